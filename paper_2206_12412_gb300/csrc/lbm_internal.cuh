// lbm_internal.cuh -- device-side data structures and launch entry points of
// the antiplane-shear lattice Boltzmann library (arXiv 2206.12412).
//
// Layout in device memory (one handle):
//   * field planes W (two ping-pong buffers) and WDOT (updated in place), each
//     (ny + 2) rows x pitch elements.  Row r = j + 1 holds lattice row j; rows
//     0 and ny + 1 are halo rows.  Each row starts with XOFF pad elements
//     (128 bytes), so lattice column 0 is 128-byte aligned and column -1 is the
//     last pad element; the right pad holds column nx.  Pads carry periodic
//     copies when an edge pair is periodic and are otherwise never used.
//     The plane pointers below point at (j = 0, i = 0).
//   * cut masks: one bit per link, ceil(nx / 32) 32-bit words per row;
//     H bit (i, j) = link (i,j)-(i+1,j), V bit (i, j) = link (i,j)-(i,j+1).
//   * rowflag[j]: bit 0 = row j has H cuts, bit 1 = row j has V cuts (links to
//     row j + 1), bit 2 = the V link row below j has cuts.  Lets the bulk
//     kernel skip the mask in the (almost all) rows without severed links.
//   * CrackState: the mutable crack and step state, read by the bulk kernel
//     (step-dependent edge values) and written by the crack kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr int kQBits = 32;                  // tip fixed point: 1 dh = 2^32 units
constexpr double kTwoM32 = 2.3283064365386963e-10;  // 2^-32
constexpr double kPi = 3.14159265358979323846;
constexpr int kBulkThreads = 128;
constexpr int kCrackThreads = 256;

enum { EDGE_FREE = 0, EDGE_DIRICHLET = 1, EDGE_PERIODIC = 2 };
enum { LEFT = 0, RIGHT = 1, BOTTOM = 2, TOP = 3 };
enum { CRACK_NONE = 0, CRACK_STATIONARY = 1, CRACK_PRESCRIBED = 2, CRACK_KCRIT = 3 };
enum { LOAD_ZERO = 0, LOAD_LINEAR = 1, LOAD_SIN2 = 2, LOAD_HALFSINE = 3, LOAD_SERIES = 4, LOAD_CONST = 5 };
enum { FLAG_CLAMPED = 1, FLAG_NONFINITE = 4 };

template <typename T> struct Pad { static constexpr int kElems = 128 / (int)sizeof(T); };

struct LoadDesc {
    int32_t kind, pad;
    double amp, t;
    const double *series;  // device copy (SERIES only)
    int64_t n;
};

// Mutable per-handle state, resident in device memory.
struct CrackState {
    int64_t step;          // completed time steps
    int64_t tip_q;         // tip x in units of 2^-32 dh
    int64_t hist_n;        // records written to the history ring
    int32_t i_first, i_last;  // severed crack links: columns i_first..i_last of V row jc-1
    int32_t arrested, flags;
    int32_t npairs, grew;
    uint32_t err_bits;     // set by the bulk kernel on a non-finite value
    int32_t pad;
    double v_prev, K, v, r_min;
    double wstar[4];       // Dirichlet values w*(t_step) for the next step
};

// Constant per-handle crack parameters (passed by value).
struct CrackParams {
    int32_t mode, jc, nx, ny;
    int32_t macro, words;
    double mu, cs, dt, dh, K_C, v_max, r0, r_min_fixed, fit_width, v_rel;
    int64_t start_q, clamp_q, hist_cap;
};

struct History {
    double *K, *v;
    int64_t *tip;
    int32_t *np;
};

template <typename T>
struct BulkArgs {
    const T *w_in;
    T *w_out;
    T *wd;
    int64_t pitch;
    int32_t nx, ny, rows;
    int32_t edge[4];
    T g, dt;
    const uint32_t *cut_h, *cut_v;
    const uint8_t *rowflag;
    int32_t words;
    CrackState *st;
};

template <typename T>
struct CrackArgs {
    const T *w_in;   // fields before the step (for the macroscopic rule)
    T *w_out;        // fields after the bulk update
    T *wd;
    int64_t pitch;
    T dt;
    CrackParams p;
    LoadDesc load[4];
    int32_t edge[4];
    uint32_t *cut_v;
    uint8_t *rowflag;
    CrackState *st;
    History hist;
};

template <typename T> cudaError_t launch_bulk(const BulkArgs<T> &a, dim3 grid, cudaStream_t s);
template <typename T> cudaError_t launch_crack(const CrackArgs<T> &a, cudaStream_t s);
cudaError_t launch_wstar(CrackState *st, const LoadDesc *load, const int32_t *edge, double dt, cudaStream_t s);
template <typename T> cudaError_t launch_fill_pads(T *w, int64_t pitch, int nx, int ny, const int32_t *edge, cudaStream_t s);

}  // namespace lbm
