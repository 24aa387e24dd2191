// lbm_internal.cuh -- device-side data structures and launch entry points of
// the antiplane-shear lattice Boltzmann library (arXiv 2206.12412).
//
// Layout in device memory (one handle):
//   * field planes W (two ping-pong buffers) and WDOT (updated in place), each
//     (ny + 2) rows x pitch elements.  Row r = j + 1 holds lattice row j; rows
//     0 and ny + 1 are halo rows.  Each row starts with XOFF pad elements
//     (128 bytes), so lattice column 0 is 128-byte aligned and column -1 is the
//     last pad element; the pad after the covered columns holds column nx.
//     After every step the pads next to free edges hold the edge sites' own
//     values (bounce-back images) and those next to periodic edges the
//     wrap-around values; pads next to Dirichlet edges are not read.  The plane pointers point at (j = 0, i = 0).
//   * cut masks: one bit per link, ceil(nx / 32) 32-bit words per row;
//     H bit (i, j) = link (i,j)-(i+1,j), V bit (i, j) = link (i,j)-(i,j+1).
//     Severed links of the crack along +x all lie in V row jc-1; the rows
//     they touch form the crack band of the step kernel's partition.  A
//     crack in any direction (line_step_kernel) severs H and V links of the
//     rows [row_lo, row_hi] of its parameters.
//   * CrackState x 2: the crack and step state, double buffered.  The step
//     kernel of step k reads buffer k & 1 and its one writer CTA writes buffer
//     (k + 1) & 1, so no CTA ever reads a state that another CTA is writing.
//   * Unit table: the row bands of the step kernel's static partition.
//   * err: sticky device error bits (non-finite field).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

constexpr int kQBits = 32;                          // tip fixed point: 1 dh = 2^32 units
constexpr double kTwoM32 = 2.3283064365386963e-10;  // 2^-32
constexpr double kPi = 3.14159265358979323846;
constexpr int kThreads = 128;                       // threads per CTA of the step kernel
constexpr int kMinBlocks = 8;                       // resident CTAs per SM the kernel is built for
constexpr int64_t kChainedSites = int64_t(1) << 18;  // lattices up to this size launch their steps chained

// EDGE_HALO: an inner edge of a row slab of a decomposed lattice; the pad
// row beyond it holds the neighbouring slab's boundary row, copied there
// after every step, and is otherwise read like any neighbour row.
enum { EDGE_FREE = 0, EDGE_DIRICHLET = 1, EDGE_PERIODIC = 2, EDGE_HALO = 3 };
enum { LEFT = 0, RIGHT = 1, BOTTOM = 2, TOP = 3 };
enum { CRACK_NONE = 0, CRACK_STATIONARY = 1, CRACK_PRESCRIBED = 2, CRACK_KCRIT = 3 };
enum { LOAD_ZERO = 0, LOAD_LINEAR = 1, LOAD_SIN2 = 2, LOAD_HALFSINE = 3, LOAD_SERIES = 4, LOAD_CONST = 5 };
enum { FLAG_CLAMPED = 1, FLAG_UNSUPPORTED = 2, FLAG_NONFINITE = 4 };
enum { ERR_NONFINITE = 1, ERR_TIMEOUT = 2 };

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream serialisation attribute (launch_chained below) may become resident
// while the kernel before it in the stream is still running.  pdl_wait()
// blocks until that kernel has completed and its memory operations are
// visible; for a kernel launched without the attribute it returns at once.
// pdl_trigger() lets the next kernel launch once every CTA of this one has
// issued it (or exited).  Every kernel of the per-step chain calls both first
// thing, before it touches memory: the next step's CTAs are then dispatched
// while this step runs and start the moment it ends, instead of after a
// launch gap and a ramp.  The next kernel launches only after every CTA of
// this one has started, so its waiting CTAs never hold a slot that one of
// this kernel's CTAs still needs.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch `kernel` on `s`, chained to the previous kernel of the stream by
// programmatic dependent launch when `chained` (the kernel must call
// pdl_wait() before it touches memory), as a plain launch otherwise.
template <typename... P, typename... A>
inline cudaError_t launch_chained(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  bool chained, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = chained ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}

// The "wdot" element type of leapfrog storage (LBM_F32_LEAPFROG): the plane it
// names is the previous w, i.e. the step's output buffer (see WdIO<Lf>).
struct Lf {
    float v;
};

template <typename T> struct Pad { static constexpr int kElems = 128 / (int)sizeof(T); };
template <typename T> struct Vec { static constexpr int N = 16 / (int)sizeof(T); };

struct LoadDesc {
    int32_t kind, pad;
    double amp, t;
    const double *series;  // device copy (SERIES only)
    int64_t n;
};

// State of one end of the crack.  decided = 1 once the crack step that
// follows LBM step `step` has been applied to this end (Alg. 1 runs after
// every LBM step); the step kernel applies a pending one before its update.
struct TipState {
    int64_t tip_q;         // tip x in units of 2^-32 dh
    int64_t tip_yq;        // tip y (a crack in any direction; else unused)
    int32_t arrested, npairs;
    int32_t grew, decided;
    int32_t flags, pad;
    double v_prev, K, v, r_min;
};

// Crack and step state after `step` LBM steps.  The right end (r) grows
// towards +x; with two-tip cracks the left end (l) grows towards -x.  Each
// end's crack step writes only its own fields (and i_last / i_first), so the
// two ends may be handled by different CTAs in the same launch.
struct CrackState {
    int64_t step;          // completed LBM steps
    int64_t hist_n;        // records written to the history ring
    int32_t i_first, i_last;  // severed crack links: columns i_first..i_last of V row jc-1
    TipState r, l;
    double wstar[4];       // Dirichlet values w*(t_step) for the next LBM step
};

// Constant per-handle crack parameters (passed by value).
struct CrackParams {
    int32_t mode, jc, nx, ny;
    int32_t macro, words;
    int32_t two_tips, q;    // q: velocity set (5 or 9)
    double mu, cs, dt, dh, K_C, v_max, r0, r_min_fixed, fit_width, v_rel;
    int64_t start_q, clamp_q, hist_cap;
    // a crack in any direction (line = 1): unit direction of growth, the
    // body's height in grid units, and the rows its severed links can touch
    int32_t line, row_lo, row_hi, band;   // band: rows of a CTA of line_step_kernel
    double dir_x, dir_y;
    int64_t clamp_yq, start_yq;
    // the crack sub-bands this lattice holds: 1 below the crack line, 2 above
    // (3: both; a row slab whose boundary is the crack line holds one)
    int32_t sides, pad_s;
    // prescribed growth: the advance v_rel c_s dt on the 2^-32 dh grid,
    // formed on the host as the crack step would form it
    int64_t dq_prescribed;
    // K-criterion growth: one unit more than the largest advance of a step,
    // v_max c_s dt on the same grid (v of eq. v-tanh never exceeds v_max)
    int64_t dq_max;
};

// Per-step records of the right end and (two-tip cracks) the left end; a
// crack in any direction records its tips' y in tipy and tipyl.
struct History {
    double *K, *v;
    int64_t *tip;
    int32_t *np;
    double *Kl, *vl;
    int64_t *tipl;
    int32_t *npl;
    int64_t *tipy, *tipyl;
};

// One row band of the static partition: output rows [j0, j1).
struct Unit {
    int32_t j0, j1, dir, pad;
};

template <typename T, typename D>
struct StepArgs {
    const T *w_in;
    T *w_out;
    D *wd;                     // wdot storage (D = T, or 16-bit with T = float)
    T wd_scale, wd_inv;        // stored value = wdot * wd_scale
    int64_t pitch;
    int32_t nx, ny;
    int32_t ncb;               // column blocks of kThreads * 16 bytes
    int32_t crack_band;        // band that holds the crack rows (-1: none)
    int32_t n_bands;           // bands of the partition
    int32_t chained;           // host side: launch chained to the previous kernel (launch_chained)
    int32_t k_cta;             // 1: the grid has one more band row (band n_bands) whose first CTA,
                               // the record CTA, runs the part of the crack step that the rows next
                               // to the crack do not wait for (prescribed growth: the K fit;
                               // K-criterion growth out of reach of a new cut: the whole step)
    int32_t edge[4];
    T g, dt;
    uint32_t *cut_h;
    uint32_t *cut_v;
    int32_t words;
    const Unit *units;
    const CrackState *s_in;
    CrackState *s_out;
    uint32_t *err;
    CrackParams p;
    LoadDesc load[4];
    History hist;
};

template <typename T>
struct FinalizeArgs {
    const T *w;
    int64_t pitch;
    CrackState *st;
    uint32_t *cut_h;
    uint32_t *cut_v;
    CrackParams p;
    History hist;
};

// One CTA of a batched step: column block cb of band `band` of lattice `inst`.
struct BatchUnit {
    int32_t inst, cb, band, pad;
};

// One piece of work of a balanced batched step (band_rows = -1): rows j0 ..
// j1 - 1 of column block cb of lattice inst, all outside its crack sub-bands,
// or (j0 < 0) the whole crack sub-band number -j0 - 1 of the lattice's band
// table.  duty: 1 = advance the step counter and the Dirichlet values of a
// lattice without a crack, 2 = write the next step's Dirichlet values of a
// lattice with one (the piece that holds the first row of the band the
// per-band launch gives that duty), 0 = none.  A CTA of the balanced step
// runs the pieces off[c] .. off[c + 1] - 1 one after another.
struct BatchPiece {
    int32_t inst;
    int16_t cb, duty;
    int32_t j0, j1;
};

// Recording of a forward run for the adjoint (see the adjoint kernel).  The
// sensors of each unit (CTA of the step kernel: band * ncb + cb) are the
// entries s_off[u] .. s_off[u+1]-1 of s_ent, each an index k into s_i / s_j.
// Step t of the recording (t = step - *n0, 0 <= t < n_steps) stores the misfit
// r = w(x_k) - target[t][k] of the state it produces in resid[t % ring][k],
// adds r^2 to loss[k] if acc_loss, and stores the first and last severed
// crack columns in force during step t in i_first[t], i_last[t].
struct RecArgs {
    const int32_t *s_off, *s_ent, *s_i, *s_j;
    const double *target;
    double *resid;
    double *loss;
    int32_t *i_first, *i_last;
    const int64_t *n0;
    int64_t n_steps, ring;
    int32_t ns, acc_loss;
};

// One step of the adjoint sweep (see lbm_adjoint.cu).  The adjoint state is
// held as the pair (m, a) in the layout of (w, wdot): m in two ping-pong
// planes with pads (w_in / w_out), a in one plane updated in place (wd).  The
// step index n is read from cnt[par] and n - 1 written to cnt[par ^ 1].
template <typename T>
struct AdjArgs {
    const T *w_in;             // m, input
    T *w_out;                  // m, output
    T *wd;                     // a
    T wd_scale, wd_inv;        // 1 (the row helpers' storage scale)
    int64_t pitch;
    int32_t nx, ny, ncb, crack_band;
    int32_t edge[4];
    T g, dt;
    int32_t jc, macro, pad0, ns;
    const Unit *units;
    const int32_t *i_first;    // [n_steps] first severed column in force during forward step t
    const int32_t *i_last;     // [n_steps] last severed column in force during forward step t
    const int64_t *cnt_in;
    int64_t *cnt_out;
    int64_t n_steps, ring;
    const int32_t *s_off, *s_ent, *s_i, *s_j;
    const double *resid;       // [ring][ns] misfits of the recorded states
    double *part;              // [n_steps][4][slots] per-CTA sums of m along the Dirichlet edges
    uint32_t *err;
    int32_t slots, pad;
};

// The grid barrier of the persistent batched kernel: arrivals of the current
// round and the round number (zeroed before a launch).
struct GridBarrier {
    unsigned int count, gen;
};

// One row copy of the halo exchange between row slabs (whole padded rows).
struct RowCopy {
    const void *src;
    void *dst;
};

// bulk: the step kernel whose interior CTAs stage rows by bulk copies (FP32 w)
template <typename T, typename D> const void *step_kernel_ptr(bool bulk = false);
// The batched step as one cooperative launch of n_steps steps (a grid
// barrier between steps, each wait bounded by `budget` clock64 cycles).
template <typename T, typename D>
cudaError_t launch_batch_persistent(const StepArgs<T, D> *descs, int n_lat, const BatchUnit *units, int n_units,
                                    const BatchUnit *eunits, int n_eunits, int par0, int64_t n_steps,
                                    GridBarrier *bar, uint32_t *err, long long budget, int threads, cudaStream_t s);
cudaError_t launch_barrier_probe(GridBarrier *bar, int ctas, int expected, long long budget, uint32_t *err,
                                 cudaStream_t s);
// threads: 32, 64 or kThreads per CTA (the batch's column-block width);
// lookahead: 1 or 2 rows of loads ahead in the march
template <typename T, typename D> cudaError_t batch_step_kernel_ptr(int threads, int lookahead, const void **fn);
template <typename T, typename D>
cudaError_t launch_batch_step(const StepArgs<T, D> *descs, const BatchUnit *units, int n_units, int par, cudaStream_t s,
                              int threads = kThreads, int lookahead = 1, bool chained = false);
// The balanced batched step: n_cta CTAs, CTA c running pieces off[c] ..
// off[c + 1] - 1.
template <typename T, typename D> cudaError_t batch_piece_kernel_ptr(int threads, int lookahead, const void **fn);
template <typename T, typename D>
cudaError_t launch_batch_pieces(const StepArgs<T, D> *descs, const BatchPiece *pieces, const int32_t *off, int n_cta,
                                int par, cudaStream_t s, int threads, int lookahead, bool chained);
template <typename T, typename D>
cudaError_t launch_step(const StepArgs<T, D> &a, int bands, cudaStream_t s, bool bulk = false);
template <typename T, typename D> cudaError_t launch_edge_rule(const StepArgs<T, D> &a, cudaStream_t s);
template <typename T, typename D> int edge_rule_count(const StepArgs<T, D> &a);
template <typename T, typename D>
cudaError_t launch_batch_edge_rule(const StepArgs<T, D> *descs, const BatchUnit *units, int n_units, int par,
                                   cudaStream_t s, bool chained = false);
template <typename T> cudaError_t launch_d2q9_step(const StepArgs<T, T> &a, cudaStream_t s);
template <typename T> cudaError_t launch_d2q9_faces(const StepArgs<T, T> &a, cudaStream_t s);
// A batch of lattices with a crack in any direction: unit (inst, cb = block
// of that lattice's line-step grid).
template <typename T, typename D>
cudaError_t launch_batch_line(const StepArgs<T, D> *descs, const BatchUnit *units, int n_units, int par, cudaStream_t s,
                              bool chained);
// A batch of D2Q9 lattices: the step units, then the crack-face units (128
// columns of one lattice with the macroscopic rule on its crack faces).
template <typename T>
cudaError_t launch_batch_d2q9(const StepArgs<T, T> *descs, const BatchUnit *units, int n_units, const BatchUnit *funits,
                             int n_funits, int par, cudaStream_t s, bool chained);
template <typename T> cudaError_t launch_step_rec(const StepArgs<T, T> &a, const RecArgs &r, int bands, cudaStream_t s);
template <typename T> const void *adjoint_kernel_ptr();
template <typename T> cudaError_t launch_adjoint(const AdjArgs<T> &a, int bands, cudaStream_t s);
cudaError_t launch_loss_sum(const double *acc, int ns, double *out, cudaStream_t s);
cudaError_t launch_grad_sum(const double *part, int64_t T, int slots, int dir_mask, double g, double *grad,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint_out(const T *a, const T *m, int64_t pitch, int nx, int ny, T dt, T *dw, T *dwd, cudaStream_t s);
template <typename D>
cudaError_t launch_wd_to_f32(const D *wd, int64_t pitch, int nx, int ny, float scale, float *dst, cudaStream_t s);
// Leapfrog storage: wdot_n = (w_n - w_{n-1}) / dt into a dense array, and
// w_{n-1} = w_n - dt wdot_n from one.
cudaError_t launch_lf_wdot(const float *w, const float *wprev, int64_t pitch, int nx, int ny, float dt, float *dst,
                           cudaStream_t s);
cudaError_t launch_lf_set_wdot(const float *w, float *wprev, int64_t pitch, int nx, int ny, float dt, const float *src,
                               cudaStream_t s);
template <typename D>
cudaError_t launch_wd_from_f32(D *wd, int64_t pitch, int nx, int ny, float scale, const float *src, cudaStream_t s);
template <typename T> cudaError_t launch_finalize(const FinalizeArgs<T> &a, cudaStream_t s);
template <typename T, typename D> cudaError_t launch_line_step(const StepArgs<T, D> &a, cudaStream_t s);
template <typename T, typename D> const void *line_step_kernel_ptr();
template <typename T> cudaError_t launch_line_finalize(const FinalizeArgs<T> &a, cudaStream_t s);
cudaError_t launch_exchange(const RowCopy *pairs, int n_pairs, int64_t row_bytes, cudaStream_t s);
cudaError_t launch_wstar(CrackState *st, const LoadDesc *load, const int32_t *edge, double dt, cudaStream_t s);
template <typename T> cudaError_t launch_fill_pads(T *w, int64_t pitch, int nx, int ny, const int32_t *edge, cudaStream_t s);

}  // namespace lbm
