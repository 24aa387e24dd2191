// lbm_host.h -- host-side state of a lattice handle and the helpers that
// the C-ABI translation units share (internal; not part of the ABI).
#pragma once

#include "lbm.h"
#include "lbm_internal.cuh"
#include "lbm_line.cuh"

typedef struct lbm_batch lbm_batch;

#include <string>
#include <type_traits>
#include <vector>

#ifndef LBM_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace lbm {
// A named range on the host timeline, for profilers (Nsight Systems, or
// ncu's --nvtx-include filters): one per C-ABI call that enqueues or waits
// for GPU work, and one per kernel family of a time step (K1 the step with
// the deferred crack step, K2 the crack-face and edge-rule solves, K3 the
// stand-alone crack step).  NVTX v3 is header-only; with no tool attached a
// range costs one indirect call.  Compile with -DLBM_NO_NVTX to drop them.
struct NvtxRange {
    explicit NvtxRange(const char *name)
    {
#ifndef LBM_NO_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange()
    {
#ifndef LBM_NO_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace lbm

using lbm::Unit;
using lbm::CrackState;
using lbm::History;
using lbm::LoadDesc;
using lbm::CrackParams;

namespace lbm {
namespace host {

// Replays runs of kernel launches that alternate between two parities as
// CUDA graphs: a ladder of graphs of kChunk, kChunk / 2, ..., 2 launches, each
// captured on first use for the starting parity it is needed at, so that a
// run of any length (a checkpoint segment of sqrt(T) steps, say) replays as
// at most one graph per level plus one single launch.
struct ChunkGraph {
    static constexpr int kLevels = 6;              // 64, 32, 16, 8, 4, 2 launches
    cudaGraphExec_t exec[kLevels][2] = {};         // [level][starting parity]
    int64_t gen = -1;
    void reset();
};

constexpr int64_t kChunk = 64;   // launches of the largest graph (every size is even: parity is kept)

}  // namespace host
}  // namespace lbm

struct lbm_handle {
    lbm_grid grid;
    lbm_lattice lat;
    lbm_material mat;
    lbm_crack crack;
    size_t esize;        // bytes per w element (and per arithmetic value)
    size_t esize_d;      // bytes per stored wdot element
    double wd_scale;     // stored wdot = wdot * wd_scale (16-bit storage)
    float *staging;      // nx * ny floats for 16-bit wdot conversions
    int64_t pitch;       // elements per padded row
    int32_t words;       // 32-bit mask words per row
    int32_t jc;          // crack line y = jc dh
    bool edge_macro;     // the macroscopic rule on the outer edges (one more kernel per step)
    int32_t q;           // velocity set: 5 or 9 (D2Q9: its own update kernel and a crack kernel per step)
    bool line;           // a straight crack in any direction (line_step_kernel)
    int32_t line_band0;  // its built-in march band height (lbm_set_launch(h, 0))
    lbm::LineFace *faces;  // its tabulated boundary points (macroscopic faces), device
    int32_t n_faces;
    double *face_scratch;  // the one-CTA face solve's scratch (lbm::FaceScratch, kLineFaceScratch bytes per point), device
    lbm::FaceChunk *face_chunks;   // the chunked face solve's tables (inside the faces allocation), device
    lbm::FaceItem *face_items;
    int32_t n_face_chunks;         // 0: the one-CTA solve
    int32_t face_solve;            // 0: chunked where the table allows, 1: always the one-CTA solve
    // step kernel shape
    int32_t ncb;         // column blocks of kThreads vectors
    int32_t n_bands, band_rows, crack_band, sms, bps;
    bool bulk;           // interior CTAs stage their rows by bulk copies (lbm_set_bulk; FP32 w, D2Q5, crack along +x)
    bool chained;        // the kernels of a step launched chained (programmatic dependent launch; lbm_set_chained)
    Unit *units;         // device table, capacity ny
    std::vector<Unit> *units_h;   // host copy of the current partition
    int64_t gen;         // bumped whenever step-kernel arguments or the partition change
    // memory
    lbm_allocator alloc;
    bool custom_alloc;
    void *block;
    size_t block_bytes;
    void *w[2];          // element (0, 0) of each W buffer
    void *wd;
    void *wbase[2], *wdbase;   // first byte of each plane (halo row, pad)
    size_t plane_bytes, plane_d_bytes;
    int64_t series_cap[4];     // capacity of each edge's device series buffer
    CrackState init_st;        // state and crack row of step 0 (lbm_reset)
    std::vector<uint32_t> *init_cut;
    uint32_t *cut_h, *cut_v;
    CrackState *st;      // two buffers
    uint32_t *err;
    History hist;
    LoadDesc load[4];
    CrackParams cp;
    double g;
    // stepping
    int parity;          // W buffer and state buffer holding the current step
    bool pending;        // the crack step after the last enqueued LBM step is not applied yet
    cudaStream_t stream;
    cudaStream_t cap_stream;
    lbm::host::ChunkGraph steps;   // graphs of runs of time steps (lbm_step)
    lbm_status sticky;
    // CUDA-event timing (lbm_set_profiling)
    int profiling;
    std::vector<cudaEvent_t> *ev;   // pairs: start, end
    std::vector<int> *ev_kind;      // 0 step kernel, 1 finalize kernel
    size_t ev_used;
    double step_ms, fin_ms;
    int64_t n_step, n_fin;
};

namespace lbm {
namespace host {

lbm_status fail(lbm_status s, const std::string &msg);
lbm_status cuda_fail(cudaError_t e, const char *what);
void clear_error();
const char *last_error();

// lbm_create; with slab = true the bottom and top edges may also be
// EDGE_HALO (inner edges of a row slab of a decomposed lattice).
// A straight crack in any direction, as lbm_create_line validated it: its
// start and initial tip on the 2^-32 dh grid, the unit direction, and the
// rows its severed links can touch.
struct LineSpec {
    int64_t start_xq, start_yq, tip_xq, tip_yq;
    double dir_x, dir_y;
    int32_t row_lo, row_hi;
};

lbm_status create_impl(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                       const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads, void *stream,
                       const lbm_allocator *allocator, bool slab, lbm_handle **out, const LineSpec *line = nullptr);

// The FP16 wdot scale lbm_create picks for these loads.
double fp16_wd_scale(const lbm_grid *grid, const lbm_loading *loads, int32_t n_loads);
// Apply the pending crack step (if any) on the handle's stream.
lbm_status finalize(lbm_handle *h);
// Synchronise, then report sticky device errors.
lbm_status check_sticky(lbm_handle *h);
// Step-kernel arguments of the step that reads W buffer `par`.
template <typename T, typename D>
inline void make_step_args(const lbm_handle *h, int par, StepArgs<T, D> &a)
{
    a.w_in = static_cast<const T *>(h->w[par]);
    a.w_out = static_cast<T *>(h->w[par ^ 1]);
    if constexpr (std::is_same<D, lbm::Lf>::value)
        a.wd = reinterpret_cast<D *>(a.w_out);   // leapfrog: w_{n-1}, overwritten by the step
    else
        a.wd = static_cast<D *>(h->wd);
    a.wd_scale = (T)h->wd_scale;
    a.wd_inv = (T)(1.0 / h->wd_scale);
    a.pitch = h->pitch;
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.ncb = h->ncb;
    a.crack_band = h->crack_band;
    a.n_bands = h->n_bands;
    a.chained = h->chained ? 1 : 0;
    a.k_cta = 0;   // set by the single-lattice launches that add the record CTA
    for (int e = 0; e < 4; ++e) { a.edge[e] = h->grid.edge[e]; a.load[e] = h->load[e]; }
    a.g = (T)h->g;
    a.dt = (T)h->grid.dt;
    a.cut_h = h->cut_h;
    a.cut_v = h->cut_v;
    a.words = h->words;
    a.units = h->units;
    a.s_in = h->st + par;
    a.s_out = h->st + (par ^ 1);
    a.err = h->err;
    a.p = h->cp;
    a.hist = h->hist;
}

// Whether the single-lattice step launch adds the record CTA (StepArgs::k_cta)
// that runs the part of a crack step the rows next to the crack do not wait
// for: the K fit of prescribed growth, or the whole step of K-criterion
// growth that cannot sever a link in it.  D2Q5 with a crack along +x, and only
// when the grid leaves a resident slot free for it, so that it runs alongside
// the first wave instead of after it.
inline bool use_k_cta(const lbm_handle *h)
{
    return (h->cp.mode == lbm::CRACK_PRESCRIBED || h->cp.mode == lbm::CRACK_KCRIT) && !h->line && h->q == 5 &&
           (int64_t)(h->n_bands + 1) * h->ncb <= (int64_t)h->sms * h->bps;
}

// Batches (lbm_batch_*): enqueue one batched step reading parity `par`; the
// common parity of the members; their state check; record n steps ending at
// parity `par`.
cudaError_t batch_enqueue(const lbm_batch *b, int par, cudaStream_t s);
int batch_parity(const lbm_batch *b);
lbm_status batch_check(const lbm_batch *b);
void batch_mark_stepped(lbm_batch *b, int par, int64_t n);


}  // namespace host
}  // namespace lbm

#define LBM_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::lbm::host::cuda_fail(e_, #call); \
    } while (0)

namespace lbm {
namespace host {

// Launch n kernels that alternate between two parities, starting at `par`:
// the largest graph of the ladder that fits, repeatedly, then one single
// launch for an odd remainder.
template <typename F>
inline lbm_status run_chunks(ChunkGraph &g, int64_t gen, cudaStream_t s, cudaStream_t cap, int64_t n, int &par, F &&enqueue)
{
    if (g.gen != gen) {
        g.reset();
        g.gen = gen;
    }
    while (n > 0) {
        int lv = 0;
        int64_t size = kChunk;
        while (lv < ChunkGraph::kLevels && size > n) {
            ++lv;
            size >>= 1;
        }
        if (lv == ChunkGraph::kLevels) {   // one launch left
            LBM_CUDA(enqueue(par, s));
            par ^= 1;
            n -= 1;
            continue;
        }
        cudaGraphExec_t &ex = g.exec[lv][par];
        if (!ex) {
            cudaGraph_t graph;
            LBM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaSuccess;
            int p = par;
            for (int64_t q = 0; q < size && ce == cudaSuccess; ++q) {
                ce = enqueue(p, cap);
                p ^= 1;
            }
            cudaError_t ee = cudaStreamEndCapture(cap, &graph);
            if (ce != cudaSuccess) return cuda_fail(ce, "capturing a step graph");
            if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
            ee = cudaGraphInstantiate(&ex, graph, 0);
            cudaGraphDestroy(graph);
            if (ee != cudaSuccess) {
                ex = nullptr;
                return cuda_fail(ee, "cudaGraphInstantiate");
            }
        }
        LBM_CUDA(cudaGraphLaunch(ex, s));
        n -= size;   // an even number of launches: the parity is kept
    }
    return LBM_OK;
}

}  // namespace host
}  // namespace lbm
