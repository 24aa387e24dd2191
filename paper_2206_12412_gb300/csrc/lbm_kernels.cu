// lbm_kernels.cu -- CUDA kernels (sm_103a) of the lattice Boltzmann time step
// for antiplane shear with dynamic mode III cracks (arXiv 2206.12412).
//
// Moment form.  With tau = dt (Sec. 3) the BGK collision sets every
// distribution to its equilibrium, f*^k = g w (k = 1..4), f*^0 = wdot - 4 g w
// (eq. f-eq, read so that sum_a f_eq^a = wdot; g = c_s^2 dt / dh^2), so the
// pair (w, wdot) is the whole state.  Streaming f*^k from the four neighbours
// and summing (eq. distrib-macro) gives
//     wdot' = wdot + g * (w_N + w_S + w_E + w_W - 4 w),     w' = w + dt wdot'
// (eq. integration), where a missing link contributes the value its boundary
// rule streams back: bounce-back f*^opp(x) = g w(x) (free edge, severed crack
// link), anti-bounce-back -f*^opp(x) + 2 g w* = g (2 w* - w(x)) (Dirichlet
// edge, Sec. 3.1), or the periodic image.  One step moves exactly 16 bytes
// per site in FP32: read w and wdot, write w and wdot.
//
// One kernel per time step.  Each CTA owns a band of rows of a 512-column
// (FP32) block and marches up through it.  The crack handling of Alg. 1 that
// follows step k - 1 is done at the start of step k by the one CTA that owns
// the next crack link (the crack band at the column of the next link); it
// reads the fields written by step k - 1 and state buffer k & 1, severs the
// link and writes state buffer (k + 1) & 1.  The macroscopic crack-face rule
// (Sec. 3.1) is applied inside the crack band, whose rows jc-3 .. jc+2 form
// a band of their own.
#include "lbm_bulk.cuh"
#include "lbm_crack.cuh"
#include "lbm_internal.cuh"
#include "lbm_rows.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <type_traits>

namespace lbm {

// ------------------------------------------------------------ step kernel
//
// Pads.  After every step the pad cell next to a free edge holds the edge
// site's own value (the bounce-back image) and the pad next to a periodic
// edge holds the wrap-around value, both written by the thread that owns the
// edge site.  Reading the pad as the neighbour then gives the boundary rule
// with no branch; only Dirichlet edges (value 2 w* - w, time dependent) and
// severed links need code of their own.
//
// Bands.  The rows are split into bands; every band except the two crack
// sub-bands runs the march below, which holds no severed link (all severed
// links of the straight crack lie between rows jc-1 and jc).  The crack
// sub-bands (rows jc-3 .. jc-1 and jc .. jc+2 with the macroscopic rule, rows
// jc-1 and jc otherwise) run crack_rows; their CTAs that own the next crack
// link first run the crack step of the previous time step.

// The fields of StepArgs that the crack sub-bands need.  Their out-of-line
// code receives them as scalars and rebuilds this struct (taking the address
// of the kernel parameter block would move all of it to local memory, and a
// struct argument copied field by field from it was not passed reliably).
template <typename T, typename D>
struct RowArgs {
    const T *w_in;
    T *w_out;
    D *wd;
    T wd_scale, wd_inv;
    int64_t pitch;
    int32_t nx, ny, jc, macro;
    int32_t edge[4];
    T g, dt;
    const uint32_t *cut_v;
    int32_t words;
    const CrackState *s_in;
};

// A crack sub-band of HH rows: rows jc-HH .. jc-1 (below the crack) or
// jc .. jc+HH-1 (above).  All of its loads are issued at once, then the rows
// are computed from registers, so the sub-band costs about one memory latency
// even while the rest of the lattice saturates HBM.  With the macroscopic
// crack-face rule (Sec. 3.1, HH = 3), the boundary point x_B next to a severed
// link takes w_B = 1.5 w_I - 0.5 w_II from the two new values of its column
// further away from the crack, and wdot(x_B) = (w_B(t+dt) - w_B(t)) / dt.
template <typename T, typename D, int HH, int TH = kThreads, bool COH = false>
__device__ __noinline__ T crack_rows(const T *w_in_, T *w_out_, D *wd_, T wd_scale_, int64_t pitch_, int nx_, int ny_,
                                     int jc_, int macro_, int edges, T g_, T dt_, const uint32_t *cut_v_, int words_,
                                     const CrackState *s_in_, int cb, int j0, int il0, int if0,
                                     const CrackState *post)
{
    RowArgs<T, D> a;
    a.w_in = w_in_;
    a.w_out = w_out_;
    a.wd = wd_;
    a.wd_scale = wd_scale_;
    a.wd_inv = (T)1 / wd_scale_;
    a.pitch = pitch_;
    a.nx = nx_;
    a.ny = ny_;
    a.jc = jc_;
    a.macro = macro_;
    for (int e = 0; e < 4; ++e) a.edge[e] = (edges >> (2 * e)) & 3;
    a.g = g_;
    a.dt = dt_;
    a.cut_v = cut_v_;
    a.words = words_;
    a.s_in = s_in_;
    T acc = (T)0;
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int x0 = (cb * TH + threadIdx.x) * N;
    const int jc = a.jc;
    const int64_t P = a.pitch;
    const T *win = a.w_in + x0;
    const bool below = j0 + HH == jc;
    R w[HH + 2], wd[HH];
    T hl[HH], hr[HH];
#pragma unroll
    for (int q = 0; q < HH + 2; ++q) load_w<COH>(win + (int64_t)(j0 - 1 + q) * P, w[q]);
#pragma unroll
    for (int q = 0; q < HH; ++q) {
        WdIO<D>::load(a.wd + x0 + (int64_t)(j0 + q) * P, wd[q], a.wd_inv);
        hl[q] = lane == 0 ? win[(int64_t)(j0 + q) * P - 1] : (T)0;
        hr[q] = lane == 31 ? win[(int64_t)(j0 + q) * P + N] : (T)0;
    }
    const EdgeValues<T> E = edge_values<T>(a.s_in);
    // the cut bits before this step's crack step (the other sub-band CTA may
    // be setting its bits meanwhile: the same bits this CTA adds below)
    const uint32_t cut0 = x0 < a.nx ? (a.cut_v[(int64_t)(jc - 1) * a.words + (x0 >> 5)] >> (x0 & 31)) & ((1u << N) - 1u) : 0u;
    __syncthreads();   // the crack step of this CTA (post != nullptr) has decided
    // the links the crack step severed: an end moves less than one spacing
    // per step, so they are the columns between the old and the new last
    // (first) severed link, (il0, i_last] on the right, [i_first, if0) on
    // the left; a CTA that ran no crack step holds none of them
    uint32_t fresh = 0u;
    if (post != nullptr) {
        const int il1 = post->i_last, if1 = post->i_first;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int i = x0 + k;
            if ((i > il0 && i <= il1) || (i >= if1 && i < if0)) fresh |= 1u << k;
        }
    }
    const uint32_t cut = x0 < a.nx ? (cut0 | fresh) : 0u;
    R o[HH], od[HH];
#pragma unroll
    for (int q = 0; q < HH; ++q) {
        const int j = j0 + q;
        T left0 = __shfl_up_sync(kFull, w[q + 1].v[N - 1], 1);
        T rightN = __shfl_down_sync(kFull, w[q + 1].v[0], 1);
        if (lane == 0) left0 = hl[q];
        if (lane == 31) rightN = hr[q];
        const uint32_t cut_up = (below && j == jc - 1) ? cut : 0u;
        const uint32_t cut_dn = (!below && j == jc) ? cut : 0u;
        row_update(a, E, x0, j, w[q + 1], w[q + 2], w[q], wd[q], left0, rightN, cut_up, cut_dn, o[q], od[q]);
    }
    if (HH >= 3 && a.macro && cut) {
        // x_B on row jc-1 (x_I, x_II on jc-2, jc-3) or on row jc (jc+1, jc+2)
        const int qb = below ? HH - 1 : 0, qi = below ? HH - 2 : 1, qii = below ? HH - 3 : 2;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if ((cut >> k) & 1u) {
                const T wB = (T)1.5 * o[qi].v[k] - (T)0.5 * o[qii].v[k];
                od[qb].v[k] = (wB - w[qb + 1].v[k]) / a.dt;
                o[qb].v[k] = wB;
            }
    }
    if (x0 < a.nx) {
#pragma unroll
        for (int q = 0; q < HH; ++q) {
            store_row(a, x0, j0 + q, o[q], od[q], acc);
            write_pads(a, x0, j0 + q, o[q]);
        }
    }
    return acc;
}

// The bulk of the lattice: a thread owns N consecutive columns (one 16-byte
// vector) of a band and marches up through it, keeping rows j-1, j, j+1 of w
// in registers, so each w value is loaded once per step (plus one halo row at
// each band end, which the neighbouring band reads at about the same time, so
// it comes from L2).  East/west neighbours come from the adjacent lanes by
// warp shuffles; lanes 0 and 31 load the halo column.  The next row's loads
// are issued before the current row is computed.  EDGE = false is the
// interior version (no edge row or column in the warp): the bare update.
template <typename T, typename D, bool EDGE, int TH = kThreads, bool COH = false, int LA = 1>
__device__ __forceinline__ void march(const StepArgs<T, D> &a, int cb, int j0, int j1, T &acc)
{
    // LA: how many rows ahead of row j + 1 the w rows (and the halo values
    // of lanes 0 and 31) are loaded: 1 keeps row j + 2 in flight while row j
    // is updated, 2 keeps rows j + 2 and j + 3 (a second row of loads in
    // flight per warp for short bands, at eight more registers)
    static_assert(LA == 1 || LA == 2, "lookahead of one or two rows");
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int x0 = (cb * TH + threadIdx.x) * N;
    const int64_t P = a.pitch;
    const T *win = a.w_in + x0;
    T *wout = a.w_out + x0;
    D *wdp = a.wd + x0;
    const T wd_inv = a.wd_inv, wd_scale = a.wd_scale;
    R wb, wc, wa, wq, wdv;
    load_w<COH>(win + (int64_t)(j0 - 1) * P, wb);
    load_w<COH>(win + (int64_t)j0 * P, wc);
    load_w<COH>(win + (int64_t)(j0 + 1) * P, wa);
    if (LA == 2 && j0 + 1 < j1) load_w<COH>(win + (int64_t)(j0 + 2) * P, wq);
    WdIO<D>::load(wdp + (int64_t)j0 * P, wdv, wd_inv);
    // wdot rows two ahead (rows j + 1 and j + 2 in flight) with a lookahead
    // of two, and for 16-bit wdot rows, which carry half the bytes of an
    // FP32 row, so that a warp has as many wdot bytes outstanding as in FP32
    constexpr bool WD2 = sizeof(D) == 2 || LA == 2;
    typename WdIO<D>::Raw wdq1;
    if (WD2 && j0 + 1 < j1) WdIO<D>::fetch(wdp + (int64_t)(j0 + 1) * P, wdq1);
    T hl = (T)0, hr = (T)0, hlq = (T)0, hrq = (T)0;
    if (lane == 0) hl = win[(int64_t)j0 * P - 1];
    if (lane == 31) hr = win[(int64_t)j0 * P + N];
    if (LA == 2 && j0 + 1 < j1) {
        if (lane == 0) hlq = win[(int64_t)(j0 + 1) * P - 1];
        if (lane == 31) hrq = win[(int64_t)(j0 + 1) * P + N];
    }
    const T g = a.g, dt = a.dt;
    EdgeValues<T> E;
    if (EDGE) E = edge_values<T>(a.s_in);
    for (int j = j0; j < j1; ++j) {
        R wn;
        typename WdIO<D>::Raw wdn;   // converted after this row's update, when it has arrived
        T hln = (T)0, hrn = (T)0;
        const bool more = j + 1 < j1;
        if (LA == 2) {
            if (j + 2 < j1) {
                load_w<COH>(win + (int64_t)(j + 3) * P, wn);
                WdIO<D>::fetch(wdp + (int64_t)(j + 2) * P, wdn);
                if (lane == 0) hln = win[(int64_t)(j + 2) * P - 1];
                if (lane == 31) hrn = win[(int64_t)(j + 2) * P + N];
            }
        } else if (more) {
            load_w<COH>(win + (int64_t)(j + 2) * P, wn);
            if (WD2) {
                if (j + 2 < j1) WdIO<D>::fetch(wdp + (int64_t)(j + 2) * P, wdn);
            } else {
                WdIO<D>::fetch(wdp + (int64_t)(j + 1) * P, wdn);
            }
            if (lane == 0) hln = win[(int64_t)(j + 1) * P - 1];
            if (lane == 31) hrn = win[(int64_t)(j + 1) * P + N];
        }
        T left0 = __shfl_up_sync(kFull, wc.v[N - 1], 1);
        T rightN = __shfl_down_sync(kFull, wc.v[0], 1);
        if (lane == 0) left0 = hl;
        if (lane == 31) rightN = hr;
        R wnew, wdnew;
        if (EDGE) {
            row_update(a, E, x0, j, wc, wa, wb, wdv, left0, rightN, 0u, 0u, wnew, wdnew);
            if (x0 < a.nx) {
                store_row(a, x0, j, wnew, wdnew, acc);
                write_pads(a, x0, j, wnew);
            }
        } else {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const T wl = k == 0 ? left0 : wc.v[k - 1];
                const T wr = k == N - 1 ? rightN : wc.v[k + 1];
                const T lap = ((wa.v[k] + wb.v[k]) + (wl + wr)) - (T)4 * wc.v[k];
                site_update<T, D>(wc.v[k], wdv.v[k], lap, g, dt, wnew.v[k], wdnew.v[k]);
            }
            stg_row(wout + (int64_t)j * P, wnew);
            WdIO<D>::store(wdp + (int64_t)j * P, wdnew, wd_scale);
            acc += wnew.v[0];
        }
        wb = wc;
        wc = wa;
        if (more) {
            if (LA == 2) {
                wa = wq;
                wq = wn;
                hl = hlq;
                hr = hrq;
                hlq = hln;
                hrq = hrn;
            } else {
                wa = wn;
                hl = hln;
                hr = hrn;
            }
            if (WD2) {
                WdIO<D>::unpack(wdq1, wdv, wd_inv);
                wdq1 = wdn;
            } else {
                WdIO<D>::unpack(wdn, wdv, wd_inv);
            }
        }
    }
}

// The bare update of an interior CTA (no edge row or column, no severed
// link) with its rows staged in shared memory by bulk asynchronous copies
// instead of per-thread loads: thread 0 keeps the copies of w rows up to
// SW - 3 = 4 ahead of the row being updated, and of wdot rows up to SD - 1
// = 4 ahead, in flight, each completing on its slot's mbarrier (16 KB per
// CTA, 130 KB per SM, whatever the number of warps), and refills the slots
// the CTA has finished with after each row.  A w slot holds the block's 512
// columns and one 16-byte vector on each side (the east / west neighbours of
// the block's edge columns).  Same arithmetic, in the same order, as the
// register march: the results are bit-identical.  Every wait gives up after
// a clock budget; then the CTA sets ERR_TIMEOUT, waits (again bounded) for
// its copies still in flight, and stops.
template <typename T, typename D>
struct BulkRing {
    static constexpr int N = Vec<T>::N;
    static constexpr int SW = 7, SD = 5;               // w slots (rows j-1, j, j+1 and 4 ahead), wdot slots
    static constexpr int WROW = kThreads * N + 2 * N;  // w elements of a slot
    static constexpr int DROW = kThreads * N;          // wdot elements of a slot
    T w[SW][WROW];
    D wd[SD][DROW];
    uint64_t bar_w[SW], bar_d[SD];
};

template <typename T, typename D>
__device__ __forceinline__ void march_bulk(const StepArgs<T, D> &a, int cb, int j0, int j1, BulkRing<T, D> &R, T &acc)
{
    typedef BulkRing<T, D> B;
    constexpr int N = Vec<T>::N;
    const unsigned kFull = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    const int xb = cb * kThreads * N;
    const int64_t P = a.pitch;
    const T *wsrc = a.w_in + xb - N;
    const D *dsrc = a.wd + xb;
    const uint32_t wbytes = B::WROW * sizeof(T), dbytes = B::DROW * sizeof(D);
    const int nw = j1 - j0 + 2;   // w rows j0 - 1 .. j1
    const int nd = j1 - j0;       // wdot rows j0 .. j1 - 1
    const long long budget = (long long)1 << 31;
    int iw = 0, id = 0;           // copies issued (thread 0)
    if (tid == 0) {
        for (int q = 0; q < B::SW; ++q) mbar_init(&R.bar_w[q]);
        for (int q = 0; q < B::SD; ++q) mbar_init(&R.bar_d[q]);
        mbar_init_fence();
        for (; iw < B::SW && iw < nw; ++iw) bulk_load(R.w[iw], wsrc + (int64_t)(j0 - 1 + iw) * P, wbytes, &R.bar_w[iw]);
        for (; id < B::SD && id < nd; ++id) bulk_load(R.wd[id], dsrc + (int64_t)(j0 + id) * P, dbytes, &R.bar_d[id]);
    }
    __syncthreads();   // the barriers are initialised before anyone waits on them
    const T g = a.g, dt = a.dt, wd_inv = a.wd_inv, wd_scale = a.wd_scale;
    T *wout = a.w_out + xb + tid * N;
    D *wdout = a.wd + xb + tid * N;
    int ok = mbar_wait(&R.bar_w[0], 0, budget) && mbar_wait(&R.bar_w[1], 0, budget);
    for (int q = 0; q < nd; ++q) {
        const int ia = q + 2;   // w index of row j + 1
        ok = ok && mbar_wait(&R.bar_w[ia % B::SW], (ia / B::SW) & 1, budget) &&
             mbar_wait(&R.bar_d[q % B::SD], (q / B::SD) & 1, budget);
        if (ok) {
            const T *rb = R.w[q % B::SW] + N + tid * N;
            const T *rc = R.w[(q + 1) % B::SW] + N + tid * N;
            const T *ra = R.w[ia % B::SW] + N + tid * N;
            Row<T, N> wb, wc, wa, wdv;
            ld_row(rb, wb);
            ld_row(rc, wc);
            ld_row(ra, wa);
            typename WdIO<D>::Raw raw;
            WdIO<D>::fetch(R.wd[q % B::SD] + tid * N, raw);
            WdIO<D>::unpack(raw, wdv, wd_inv);
            T left0 = __shfl_up_sync(kFull, wc.v[N - 1], 1);
            T rightN = __shfl_down_sync(kFull, wc.v[0], 1);
            if (lane == 0) left0 = rc[-1];
            if (lane == 31) rightN = rc[N];
            Row<T, N> wnew, wdnew;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const T wl = k == 0 ? left0 : wc.v[k - 1];
                const T wr = k == N - 1 ? rightN : wc.v[k + 1];
                const T lap = ((wa.v[k] + wb.v[k]) + (wl + wr)) - (T)4 * wc.v[k];
                site_update<T, D>(wc.v[k], wdv.v[k], lap, g, dt, wnew.v[k], wdnew.v[k]);
            }
            const int64_t o = (int64_t)(j0 + q) * P;
            stg_row(wout + o, wnew);
            WdIO<D>::store(wdout + o, wdnew, wd_scale);
            acc += wnew.v[0];
        }
        // every thread is done with w row j - 1 and wdot row j: refill their slots
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) {
            if (iw < nw) {
                bulk_load(R.w[iw % B::SW], wsrc + (int64_t)(j0 - 1 + iw) * P, wbytes, &R.bar_w[iw % B::SW]);
                ++iw;
            }
            if (id < nd) {
                bulk_load(R.wd[id % B::SD], dsrc + (int64_t)(j0 + id) * P, dbytes, &R.bar_d[id % B::SD]);
                ++id;
            }
        }
    }
    if (!ok) {
        // a copy did not arrive within the budget: report it, and let the
        // copies still in flight land (bounded) before the CTA leaves
        if (tid == 0) {
            atomicOr(a.err, (uint32_t)ERR_TIMEOUT);
            for (int q = 0; q < B::SW && q < iw; ++q) {
                const int last = q + B::SW * ((iw - 1 - q) / B::SW);
                mbar_wait(&R.bar_w[q], (last / B::SW) & 1, budget);
            }
            for (int q = 0; q < B::SD && q < id; ++q) {
                const int last = q + B::SD * ((id - 1 - q) / B::SD);
                mbar_wait(&R.bar_d[q], (last / B::SD) & 1, budget);
            }
        }
        __syncthreads();
    }
}

// A lattice without a crack: only the step counter and the Dirichlet values
// advance (one thread of the CTA that holds band 0, column block 0).
template <typename T, typename D>
__device__ __forceinline__ void advance_without_crack(const StepArgs<T, D> &a, CrackState &sS)
{
    sS = *a.s_in;
    const int64_t n = sS.step + 1;
    sS.step = n;
    sS.r.decided = 1;
    sS.l.decided = 1;
    for (int e = 0; e < 4; ++e)
        sS.wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)a.p.dt) : 0.0;
    *a.s_out = sS;
}

// A lattice with a crack: the Dirichlet values w*(t_{n+1}) of the next step
// (its own fields of the next state; the crack step's writer CTA writes the
// others).
template <typename T, typename D>
__device__ __forceinline__ void next_dirichlet_values(const StepArgs<T, D> &a)
{
    const int64_t n = a.s_in->step + 1;
    for (int e = 0; e < 4; ++e)
        a.s_out->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)a.p.dt) : 0.0;
}

// One CTA of a time step: column block cb of band `band` of the lattice that
// `a` describes (the kernel parameter block, or a copy in shared memory).
// BOTH: compiled with the path that evaluates the two ends of a two-tip
// crack at once when one CTA holds both (kept out of the single-tip
// kernels, whose march it slows through the larger kernel).
// TH: threads of the CTA (a column block is TH 16-byte vectors wide); the
// single-lattice kernels use kThreads, the batched kernel any multiple of 32.
// COH: w read with coherent loads (the persistent batched kernel, where the
// same launch wrote it).
// ring: the shared-memory ring of the bulk march (nullptr: every CTA takes
// the register march).
template <typename T, typename D, bool REC, bool BOTH = false, int TH = kThreads, bool COH = false, int LA = 1>
__device__ __forceinline__ void step_cta(const StepArgs<T, D> &a, int cb, int band, CrackState &sS, const RecArgs &r,
                                         BulkRing<T, D> *ring = nullptr)
{
    constexpr int N = Vec<T>::N;
    const unsigned kFull = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    const CrackParams &p = a.p;
    if (a.k_cta && band == a.n_bands) {
        // the record CTA (band n_bands has no unit), at the same time as the
        // crack sub-bands update their rows: for prescribed growth the K fit
        // for the history (warp 0 the right end, warp 1 the left one) while
        // the sub-bands advance the tip; for K-criterion growth that cannot
        // sever a link in this step the whole crack step
        if (cb == 0) {
            if (tid == 0) sS = *a.s_in;
            __syncthreads();
            if (p.mode == CRACK_PRESCRIBED) {
                if (tid < 32)
                    crack_record_prescribed<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, a.s_out, a.err, +1);
                else if (tid < 64 && p.two_tips)
                    crack_record_prescribed<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, a.s_out, a.err, -1);
            } else if (p.mode == CRACK_KCRIT && !REC && !crack_cut_in_reach(p, sS)) {
                // K-criterion growth that cannot sever a link in this step:
                // the whole crack step here, by the warps the crack sub-band
                // CTAs would run it with (the same sums in the same order),
                // while those CTAs update their rows
                constexpr int cols = TH * Vec<T>::N;
                int i_next = max(sS.i_last + 1, sS.i_first);
                i_next = min(max(i_next, 0), a.nx - 1);
                int i_prev = min(sS.i_first - 1, sS.i_last);
                i_prev = min(max(i_prev, 0), a.nx - 1);
                const bool pending = !sS.r.decided;
                if (BOTH && p.two_tips && i_next / cols == i_prev / cols) {
                    if (tid < 32) crack_step_both<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, true);
                } else if (tid < 32) {
                    crack_step_warp<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, +1, true);
                } else if (tid < 64 && p.two_tips) {
                    crack_step_warp<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, -1, true);
                }
                __syncthreads();
                if (tid == 0) {
                    CrackState *o = a.s_out;
                    const int64_t n = sS.step + 1;
                    o->step = n;
                    o->hist_n = sS.hist_n + (pending ? 1 : 0);
                    o->i_last = sS.i_last;
                    o->i_first = sS.i_first;
                    o->r = sS.r;
                    o->r.decided = 0;
                    if (p.two_tips) {
                        o->l = sS.l;
                        o->l.decided = 0;
                    }
                    if (a.n_bands <= 2)
                        for (int e = 0; e < 4; ++e)
                            o->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)p.dt) : 0.0;
                }
            }
        }
        return;
    }
    const Unit U = a.units[band];
    const int j0 = U.j0, j1 = U.j1;
    const int nx = a.nx;
    T acc = (T)0;
    // prescribed growth with a record CTA: the crack sub-bands only advance
    const bool rec_elsewhere = a.k_cta && p.mode == CRACK_PRESCRIBED;

    if (a.crack_band >= 0 && (band == a.crack_band || (band == a.crack_band + 1 && p.sides == 3))) {
        // The crack step of Alg. 1 that follows the previous LBM step, by the
        // two crack sub-band CTAs that own the next link of each end: both
        // reach the same decision; the lower one records it, each end
        // writing only its own fields of the next state.  (A row slab whose
        // boundary is the crack line holds one of the two sub-bands and
        // reads the other side's row from its halo: it records its own.)
        const int cols = TH * N;
        // the state, for the crack step, loaded at once with the two fields
        // every thread reads (an unused copy where no end is in this CTA)
        if (tid == 0) sS = *a.s_in;
        const int il0 = a.s_in->i_last, if0 = a.s_in->i_first;   // before the crack step
        int i_next = il0 + 1;
        i_next = max(i_next, if0);
        i_next = min(max(i_next, 0), nx - 1);
        int i_prev = if0 - 1;
        i_prev = min(i_prev, il0);
        i_prev = min(max(i_prev, 0), nx - 1);
        const bool right_here = cb == i_next / cols;
        const bool left_here = p.two_tips && cb == i_prev / cols;
        const bool commit = band == a.crack_band;
        const bool both = BOTH && right_here && left_here;
        if ((right_here || left_here) && tid == 0 && !rec_elsewhere) {
            // the rows this CTA updates after the crack step, brought into L2
            // while the crack step runs (its FP64 chain is the long pole)
            const int hh = p.macro ? 3 : 1;
            const int64_t xb = (int64_t)cb * TH * N;
            for (int q = -1; q <= hh; ++q)
                bulk_prefetch_l2(a.w_in + (int64_t)(j0 + q) * a.pitch + xb, (uint32_t)(TH * N * sizeof(T)));
            for (int q = 0; q < hh; ++q)
                bulk_prefetch_l2(a.wd + (int64_t)(j0 + q) * a.pitch + xb, (uint32_t)(TH * N * sizeof(D)));
        }
        // K-criterion growth that cannot sever a link in this step: the
        // record CTA runs the whole crack step; this CTA's rows need no
        // decision (sS keeps the severed columns of s_in: no fresh cut)
        bool kc_elsewhere = false;
        if ((right_here || left_here) && tid < 32 && a.k_cta && p.mode == CRACK_KCRIT && !REC) {
            __syncwarp();
            kc_elsewhere = !crack_cut_in_reach(p, sS);
        }
        if ((right_here || left_here) && tid < 32 && !kc_elsewhere) {
            __syncwarp();
            const bool pending = !sS.r.decided;   // not yet applied by a deferred crack step
            if (rec_elsewhere) {
                // the advance needs no K: lane 0 advances each end here (the
                // right end first, as below), the record CTA forms K
                if (tid == 0) {
                    if (right_here) crack_advance_prescribed(p, a.cut_v, a.hist, sS, +1, commit);
                    if (left_here) crack_advance_prescribed(p, a.cut_v, a.hist, sS, -1, commit);
                }
                __syncwarp();
            } else if (both) {
                // both ends in this CTA: their criteria at once, then the
                // right end's advance and the left end's
                crack_step_both<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, commit);
            } else {
                if (right_here) crack_step_warp<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, +1, commit);
                if (left_here) crack_step_warp<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, -1, commit);
            }
            if (tid == 0 && commit) {
                CrackState *o = a.s_out;
                const int64_t n = sS.step + 1;
                if (right_here) {
                    o->step = n;
                    o->hist_n = sS.hist_n + (pending ? 1 : 0);
                    o->i_last = sS.i_last;
                    if (!p.two_tips) o->i_first = sS.i_first;
                    if (rec_elsewhere) copy_tip_decision(o->r, sS.r);   // K, r_min, npairs: the record CTA
                    else o->r = sS.r;
                    o->r.decided = 0;
                    // the Dirichlet values of the next step come from another
                    // CTA when there is one (see below): their FP64 sin of the
                    // sin^2 and half-sine loads stays off this CTA's path
                    if (a.n_bands <= 2)
                        for (int e = 0; e < 4; ++e)
                            o->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)p.dt) : 0.0;
                }
                if (left_here) {
                    o->i_first = sS.i_first;
                    if (rec_elsewhere) copy_tip_decision(o->l, sS.l);
                    else o->l = sS.l;
                    o->l.decided = 0;
                }
                if (REC) {
                    const int64_t t = n - 1 - *r.n0;
                    if (t >= 0 && t < r.n_steps) {
                        if (right_here) r.i_last[t] = sS.i_last;
                        if (right_here && !p.two_tips) r.i_first[t] = sS.i_first;
                        if (left_here) r.i_first[t] = sS.i_first;
                    }
                }
            }
        }
        const int edges = a.edge[0] | (a.edge[1] << 2) | (a.edge[2] << 4) | (a.edge[3] << 6);
        const CrackState *post = (right_here || left_here) ? &sS : nullptr;
        acc = p.macro ? crack_rows<T, D, 3, TH, COH>(a.w_in, a.w_out, a.wd, a.wd_scale, a.pitch, a.nx, a.ny, p.jc,
                                                p.macro, edges, a.g, a.dt, a.cut_v, a.words, a.s_in, cb, j0, il0,
                                                if0, post)
                      : crack_rows<T, D, 1, TH, COH>(a.w_in, a.w_out, a.wd, a.wd_scale, a.pitch, a.nx, a.ny, p.jc,
                                                p.macro, edges, a.g, a.dt, a.cut_v, a.words, a.s_in, cb, j0, il0,
                                                if0, post);
    } else {
        if (a.crack_band < 0 && cb == 0 && band == 0 && tid == 0) advance_without_crack(a, sS);
        // the edge rules per warp: only warps whose columns reach an outer edge,
        // and the bands holding the bottom and top rows, need them
        const int xw0 = (cb * TH + (tid & ~31)) * N;   // first column of this warp
        const bool edge = (xw0 == 0) | (xw0 + 32 * N - 1 >= nx - 1) | (j0 == 0) | (j1 == a.ny);
        // a CTA with no edge row or column anywhere takes the bulk march
        // when there is a ring (uniform across the CTA: its barriers)
        const int xb = cb * TH * N;
        const bool inner = xb > 0 && xb + TH * N < nx && j0 > 0 && j1 < a.ny;
        if (ring != nullptr && TH == kThreads && inner) {
            march_bulk<T, D>(a, cb, j0, j1, *ring, acc);
        } else if (xw0 < nx) {
            // warps wholly right of the lattice (the ragged last column block)
            // have nothing to load or store
            if (edge) march<T, D, true, TH, COH, LA>(a, cb, j0, j1, acc);
            else march<T, D, false, TH, COH, LA>(a, cb, j0, j1, acc);
        }
    }
    // with a crack, the Dirichlet values w*(t_{n+1}) of the next step are
    // written by the first CTA of the first band that is no crack sub-band
    // (its own fields of the next state; the writer CTA writes the others)
    if (a.crack_band >= 0 && a.n_bands > 2 && cb == 0 && tid == 0 &&
        band == (a.crack_band > 0 ? 0 : a.crack_band + (p.sides == 3 ? 2 : 1)))
        next_dirichlet_values(a);
    // a non-finite w (or wdot, which enters w) turns the sum of the first
    // component of each vector non-finite within a step or two
    if (__any_sync(kFull, !isfinite(acc)) && lane == 0) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
    if (REC) {
        // the sensors this CTA owns: misfit of the new state (its own stores
        // are visible to the CTA after the barrier)
        __syncthreads();
        const int64_t t = a.s_in->step - *r.n0;
        if (t >= 0 && t < r.n_steps) {
            // one thread per sensor of the list (each sensor appears once)
            const int u = band * a.ncb + cb;
            const int lo = r.s_off[u], hi = r.s_off[u + 1];
            for (int q = lo + tid; q < hi; q += TH) {
                const int k = r.s_ent[q];
                const double wv = (double)a.w_out[(int64_t)r.s_j[k] * a.pitch + r.s_i[k]];
                const double res = wv - r.target[t * r.ns + k];
                r.resid[(t % r.ring) * r.ns + k] = res;
                if (r.acc_loss) r.loss[k] += res * res;
            }
        }
    }
}

template <typename T, typename D, bool BOTH>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2) step_kernel(const StepArgs<T, D> a)
{
    __shared__ CrackState sS;
    pdl_wait();
    pdl_trigger();
    step_cta<T, D, false, BOTH>(a, blockIdx.x, blockIdx.y, sS, RecArgs{});
}

// The step kernel whose interior CTAs stage their rows with bulk copies
// (FP32 w; see march_bulk).
template <typename T, typename D, bool BOTH>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_kernel_bulk(const StepArgs<T, D> a)
{
    __shared__ CrackState sS;
    __shared__ __align__(128) BulkRing<T, D> ring;
    pdl_wait();
    pdl_trigger();
    step_cta<T, D, false, BOTH>(a, blockIdx.x, blockIdx.y, sS, RecArgs{}, &ring);
}

// The step kernel with the recording of a forward run for the adjoint.
template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2)
    step_rec_kernel(const StepArgs<T, T> a, const RecArgs r)
{
    __shared__ CrackState sS;
    step_cta<T, T, true>(a, blockIdx.x, blockIdx.y, sS, r);
}

// Many independent lattices in one launch: CTA u runs unit u of the batch,
// with its lattice's arguments (for the current parity) copied to shared
// memory first.  TH threads per CTA: the column blocks of a batch are TH
// vectors wide (TH * 4 FP32 columns), chosen per batch (lbm_batch_tune) so
// that few warps fall right of their lattice.  Occupancy is register bound
// at 64 registers, i.e. the same 32 warps per SM for every TH.  LA: the
// march's lookahead in rows; two rows take eight more registers (28 warps
// per SM) for twice the loads in flight per warp.
template <typename T, typename D, int TH, int LA>
__global__ void __launch_bounds__(TH, (sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2) * (kThreads / TH) -
                                          (LA == 2 ? kThreads / TH : 0))
    batch_step_kernel(const StepArgs<T, D> *descs, const BatchUnit *units, int par)
{
    __shared__ CrackState sS;
    __shared__ __align__(16) StepArgs<T, D> sa;
    pdl_wait();
    pdl_trigger();
    const BatchUnit u = units[blockIdx.x];
    const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + 2 * u.inst + par);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
    for (int q = threadIdx.x; q < (int)(sizeof(StepArgs<T, D>) / 4); q += TH) dst[q] = src[q];
    __syncthreads();
    step_cta<T, D, false, false, TH, false, LA>(sa, u.cb, u.band, sS, RecArgs{});
}

// The balanced batched step (band_rows = -1): as many CTAs as are resident at
// once, each running a list of pieces (BatchPiece) chosen on the host so that
// every CTA has about the same number of rows to march, whatever the
// lattices' heights: a crack sub-band runs the per-band code, any other piece
// marches its rows exactly as the band that holds them would (the same per-
// warp edge handling, the same per-site arithmetic), so the results are
// bit-identical to the per-band launch.  One wave, no tail of short units,
// and long marches with few halo rows.
template <typename T, typename D, int TH, int LA>
__device__ __forceinline__ void piece_rows(const StepArgs<T, D> &a, int cb, int j0, int j1, int duty, CrackState &sS)
{
    constexpr int N = Vec<T>::N;
    const int tid = threadIdx.x;
    T acc = (T)0;
    if (duty == 1 && tid == 0) advance_without_crack(a, sS);
    if (duty == 2 && tid == 0) next_dirichlet_values(a);
    const int xw0 = (cb * TH + (tid & ~31)) * N;   // first column of this warp
    if (xw0 < a.nx) {
        if ((xw0 == 0) | (xw0 + 32 * N - 1 >= a.nx - 1)) {
            march<T, D, true, TH, false, LA>(a, cb, j0, j1, acc);
        } else {
            // the bottom and top rows of the lattice take the edge rules, the
            // rows between them the bare update (a piece is often a long run
            // from an outer edge)
            const int lo = j0 == 0 ? 1 : j0, hi = j1 == a.ny ? a.ny - 1 : j1;
            if (j0 == 0) march<T, D, true, TH, false, LA>(a, cb, 0, 1, acc);
            if (lo < hi) march<T, D, false, TH, false, LA>(a, cb, lo, hi, acc);
            if (j1 == a.ny && a.ny - 1 >= lo) march<T, D, true, TH, false, LA>(a, cb, a.ny - 1, a.ny, acc);
        }
    }
    if (__any_sync(0xffffffffu, !isfinite(acc)) && (tid & 31) == 0) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
}

template <typename T, typename D, int TH, int LA>
__global__ void __launch_bounds__(TH, (sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2) * (kThreads / TH) -
                                          (LA == 2 ? kThreads / TH : 0))
    batch_piece_kernel(const StepArgs<T, D> *descs, const BatchPiece *pieces, const int32_t *off, int par)
{
    __shared__ CrackState sS;
    __shared__ __align__(16) StepArgs<T, D> sa;
    pdl_wait();
    pdl_trigger();
    const int q0 = off[blockIdx.x], q1 = off[blockIdx.x + 1];
    int cur = -1;
    for (int q = q0; q < q1; ++q) {
        const BatchPiece u = pieces[q];
        // every thread is done with the previous piece (its arguments, sS)
        if (q > q0) __syncthreads();
        if (u.inst != cur) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + 2 * u.inst + par);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
            for (int k = threadIdx.x; k < (int)(sizeof(StepArgs<T, D>) / 4); k += TH) dst[k] = src[k];
            __syncthreads();
            cur = u.inst;
        }
        if (u.j0 < 0) step_cta<T, D, false, false, TH, false, LA>(sa, u.cb, -u.j0 - 1, sS, RecArgs{});
        else piece_rows<T, D, TH, LA>(sa, u.cb, u.j0, u.j1, u.duty, sS);
    }
}

// ----------------------------------------- persistent batched step
//
// One cooperative launch advances every lattice of a batch by n steps: each
// CTA takes the units u = blockIdx.x, blockIdx.x + gridDim.x, ... of a step,
// then all CTAs meet at a grid barrier before the next step (and between a
// step and its edge-rule units).  The wait at the barrier is bounded: after
// `budget` clock64 cycles a CTA sets ERR_TIMEOUT in the batch's error word
// and in every lattice's, and returns; the others then give up at their next
// wait (they see the flag), so the launch always ends.  w is read with
// coherent loads, since the launch itself wrote the previous step's w.

template <typename T, typename D>
__device__ __forceinline__ void edge_rule_at(const StepArgs<T, D> &a, int t);

// Arrive and wait until `expected` CTAs have arrived (bounded).  Returns
// false (and sets ERR_TIMEOUT in *err) if the wait gave up.
__device__ __forceinline__ bool grid_barrier(GridBarrier *bar, unsigned expected, long long budget, uint32_t *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *vg = &bar->gen;
        volatile uint32_t *ve = err;
        const unsigned g = *vg;
        __threadfence();   // this CTA's stores (ordered by the CTA barrier) before the arrival
        if (atomicAdd(&bar->count, 1u) == expected - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vg == g) {
                if ((*ve & ERR_TIMEOUT) || clock64() - t0 > budget) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();   // the other CTAs' stores before this CTA's next loads
        if (!ok) atomicOr(err, (uint32_t)ERR_TIMEOUT);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T, typename D>
__device__ void flag_timeout(const StepArgs<T, D> *descs, int n_lat)
{
    for (int i = threadIdx.x; i < n_lat; i += blockDim.x) atomicOr(descs[2 * i].err, (uint32_t)ERR_TIMEOUT);
}

template <typename T, typename D, int TH>
__global__ void __launch_bounds__(TH, (sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2) * (kThreads / TH))
    batch_persistent_kernel(const StepArgs<T, D> *descs, int n_lat, const BatchUnit *units, int n_units,
                            const BatchUnit *eunits, int n_eunits, int par0, int64_t n_steps, GridBarrier *bar,
                            uint32_t *err, long long budget)
{
    __shared__ CrackState sS;
    __shared__ __align__(16) StepArgs<T, D> sa;
    const unsigned nb = gridDim.x;
    for (int64_t k = 0; k < n_steps; ++k) {
        const int par = par0 ^ (int)(k & 1);
        for (int q = blockIdx.x; q < n_units; q += nb) {
            const BatchUnit u = units[q];
            const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + 2 * u.inst + par);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
            __syncthreads();   // the previous unit is done with sa and sS
            for (int t = threadIdx.x; t < (int)(sizeof(StepArgs<T, D>) / 4); t += TH) dst[t] = src[t];
            __syncthreads();
            step_cta<T, D, false, false, TH, true>(sa, u.cb, u.band, sS, RecArgs{});
        }
        if (n_eunits > 0) {
            if (!grid_barrier(bar, nb, budget, err)) {
                flag_timeout(descs, n_lat);
                return;
            }
            for (int q = blockIdx.x; q < n_eunits; q += nb) {
                const BatchUnit u = eunits[q];
                for (int t = threadIdx.x; t < 128; t += TH) edge_rule_at(descs[2 * u.inst + par], u.cb + t);
            }
        }
        if (!grid_barrier(bar, nb, budget, err)) {
            flag_timeout(descs, n_lat);
            return;
        }
    }
}

// A diagnostic of the bounded wait: `ctas` CTAs meet at a barrier that
// expects `expected` arrivals; with fewer CTAs than expected nothing
// completes it and every wait gives up after `budget` cycles.
__global__ void barrier_probe_kernel(GridBarrier *bar, unsigned expected, long long budget, uint32_t *err)
{
    grid_barrier(bar, expected, budget, err);
}

cudaError_t launch_barrier_probe(GridBarrier *bar, int ctas, int expected, long long budget, uint32_t *err,
                                 cudaStream_t s)
{
    barrier_probe_kernel<<<(unsigned)ctas, 32, 0, s>>>(bar, (unsigned)expected, budget, err);
    return cudaGetLastError();
}

template <typename T, typename D>
cudaError_t persistent_grid(int threads, int n_units, int *grid)
{
    const void *fn = nullptr;
    switch (threads) {
    case 32: fn = reinterpret_cast<const void *>(&batch_persistent_kernel<T, D, 32>); break;
    case 64: fn = reinterpret_cast<const void *>(&batch_persistent_kernel<T, D, 64>); break;
    case kThreads: fn = reinterpret_cast<const void *>(&batch_persistent_kernel<T, D, kThreads>); break;
    default: return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, 0);
    if (e != cudaSuccess) return e;
    const int cap = sms * bps;
    *grid = n_units < cap ? n_units : cap;
    return *grid > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <typename T, typename D>
cudaError_t launch_batch_persistent(const StepArgs<T, D> *descs, int n_lat, const BatchUnit *units, int n_units,
                                    const BatchUnit *eunits, int n_eunits, int par0, int64_t n_steps,
                                    GridBarrier *bar, uint32_t *err, long long budget, int threads, cudaStream_t s)
{
    int grid = 0;
    cudaError_t e = persistent_grid<T, D>(threads, n_units, &grid);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&descs, (void *)&n_lat, (void *)&units, (void *)&n_units, (void *)&eunits,
                    (void *)&n_eunits, (void *)&par0, (void *)&n_steps, (void *)&bar, (void *)&err, (void *)&budget};
    const void *fn = threads == 32 ? reinterpret_cast<const void *>(&batch_persistent_kernel<T, D, 32>)
                   : threads == 64 ? reinterpret_cast<const void *>(&batch_persistent_kernel<T, D, 64>)
                                   : reinterpret_cast<const void *>(&batch_persistent_kernel<T, D, kThreads>);
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3((unsigned)threads), args, 0, s);
}

template <typename T, typename D> const void *step_kernel_ptr(bool bulk)
{
    if constexpr (sizeof(T) == 4)
        if (bulk) return reinterpret_cast<const void *>(&step_kernel_bulk<T, D, false>);
    return reinterpret_cast<const void *>(&step_kernel<T, D, false>);
}

template <typename T, typename D>
cudaError_t launch_step(const StepArgs<T, D> &a, int bands, cudaStream_t s, bool bulk)
{
    const dim3 grid((unsigned)a.ncb, (unsigned)(bands + (a.k_cta ? 1 : 0)));
    const bool ch = a.chained != 0;
    if constexpr (sizeof(T) == 4) {
        if (bulk)
            return a.p.two_tips ? launch_chained(step_kernel_bulk<T, D, true>, grid, dim3(kThreads), 0, s, ch, a)
                                : launch_chained(step_kernel_bulk<T, D, false>, grid, dim3(kThreads), 0, s, ch, a);
    }
    return a.p.two_tips ? launch_chained(step_kernel<T, D, true>, grid, dim3(kThreads), 0, s, ch, a)
                        : launch_chained(step_kernel<T, D, false>, grid, dim3(kThreads), 0, s, ch, a);
}

template <typename T>
cudaError_t launch_step_rec(const StepArgs<T, T> &a, const RecArgs &r, int bands, cudaStream_t s)
{
    step_rec_kernel<T><<<dim3((unsigned)a.ncb, (unsigned)(bands + (a.k_cta ? 1 : 0))), kThreads, 0, s>>>(a, r);
    return cudaGetLastError();
}

template <typename T, typename D>
cudaError_t batch_step_kernel_ptr(int threads, int lookahead, const void **fn)
{
    const bool deep = lookahead == 2;
    if (lookahead != 1 && !deep) return cudaErrorInvalidValue;
    switch (threads) {
    case 32:
        *fn = deep ? reinterpret_cast<const void *>(&batch_step_kernel<T, D, 32, 2>)
                   : reinterpret_cast<const void *>(&batch_step_kernel<T, D, 32, 1>);
        return cudaSuccess;
    case 64:
        *fn = deep ? reinterpret_cast<const void *>(&batch_step_kernel<T, D, 64, 2>)
                   : reinterpret_cast<const void *>(&batch_step_kernel<T, D, 64, 1>);
        return cudaSuccess;
    case kThreads:
        *fn = deep ? reinterpret_cast<const void *>(&batch_step_kernel<T, D, kThreads, 2>)
                   : reinterpret_cast<const void *>(&batch_step_kernel<T, D, kThreads, 1>);
        return cudaSuccess;
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, typename D>
cudaError_t launch_batch_step(const StepArgs<T, D> *descs, const BatchUnit *units, int n_units, int par, cudaStream_t s,
                              int threads, int lookahead, bool chained)
{
    const void *fn = nullptr;
    cudaError_t e = batch_step_kernel_ptr<T, D>(threads, lookahead, &fn);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&descs, (void *)&units, (void *)&par};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_units);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = chained ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

template <typename T, typename D>
cudaError_t batch_piece_kernel_ptr(int threads, int lookahead, const void **fn)
{
    const bool deep = lookahead == 2;
    if (lookahead != 1 && !deep) return cudaErrorInvalidValue;
    switch (threads) {
    case 32:
        *fn = deep ? reinterpret_cast<const void *>(&batch_piece_kernel<T, D, 32, 2>)
                   : reinterpret_cast<const void *>(&batch_piece_kernel<T, D, 32, 1>);
        return cudaSuccess;
    case 64:
        *fn = deep ? reinterpret_cast<const void *>(&batch_piece_kernel<T, D, 64, 2>)
                   : reinterpret_cast<const void *>(&batch_piece_kernel<T, D, 64, 1>);
        return cudaSuccess;
    case kThreads:
        *fn = deep ? reinterpret_cast<const void *>(&batch_piece_kernel<T, D, kThreads, 2>)
                   : reinterpret_cast<const void *>(&batch_piece_kernel<T, D, kThreads, 1>);
        return cudaSuccess;
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, typename D>
cudaError_t launch_batch_pieces(const StepArgs<T, D> *descs, const BatchPiece *pieces, const int32_t *off, int n_cta,
                                int par, cudaStream_t s, int threads, int lookahead, bool chained)
{
    const void *fn = nullptr;
    cudaError_t e = batch_piece_kernel_ptr<T, D>(threads, lookahead, &fn);
    if (e != cudaSuccess) return e;
    if (n_cta <= 0) return cudaSuccess;
    void *args[] = {(void *)&descs, (void *)&pieces, (void *)&off, (void *)&par};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_cta);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = chained ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// ------------------------------------------ wdot planes in 16-bit storage

template <typename D>
__global__ void wd_to_f32_kernel(const D *wd, int64_t P, int nx, int ny, float inv, float *dst)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nx * ny) return;
    const int j = (int)(t / nx), i = (int)(t % nx);
    dst[t] = WdIO<D>::get(wd + (int64_t)j * P + i, inv);
}

template <typename D>
__global__ void wd_from_f32_kernel(D *wd, int64_t P, int nx, int ny, float scale, const float *src)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nx * ny) return;
    const int j = (int)(t / nx), i = (int)(t % nx);
    WdIO<D>::put(wd + (int64_t)j * P + i, src[t], scale);
}

template <typename D>
cudaError_t launch_wd_to_f32(const D *wd, int64_t pitch, int nx, int ny, float scale, float *dst, cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny;
    wd_to_f32_kernel<D><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(wd, pitch, nx, ny, 1.0f / scale, dst);
    return cudaGetLastError();
}

template <typename D>
cudaError_t launch_wd_from_f32(D *wd, int64_t pitch, int nx, int ny, float scale, const float *src, cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny;
    wd_from_f32_kernel<D><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(wd, pitch, nx, ny, scale, src);
    return cudaGetLastError();
}

// --------------------------------------------- leapfrog storage: wdot

__global__ void lf_wdot_kernel(const float *w, const float *wprev, int64_t P, int nx, int ny, float dt, float *dst)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nx * ny) return;
    const int64_t o = (t / nx) * P + t % nx;
    dst[t] = (w[o] - wprev[o]) / dt;
}

__global__ void lf_set_wdot_kernel(const float *w, float *wprev, int64_t P, int nx, int ny, float dt, const float *src)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nx * ny) return;
    const int64_t o = (t / nx) * P + t % nx;
    wprev[o] = w[o] - dt * src[t];
}

cudaError_t launch_lf_wdot(const float *w, const float *wprev, int64_t pitch, int nx, int ny, float dt, float *dst,
                           cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny;
    lf_wdot_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, wprev, pitch, nx, ny, dt, dst);
    return cudaGetLastError();
}

cudaError_t launch_lf_set_wdot(const float *w, float *wprev, int64_t pitch, int nx, int ny, float dt, const float *src,
                               cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny;
    lf_set_wdot_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, wprev, pitch, nx, ny, dt, src);
    return cudaGetLastError();
}

// ----------------------------------------------------- pending crack step

// The crack step that follows the last enqueued LBM step, applied in place
// before the host reads the state (one warp).
template <typename T>
__global__ void finalize_kernel(const FinalizeArgs<T> a)
{
    __shared__ CrackState sS;
    if (threadIdx.x == 0) sS = *a.st;
    __syncwarp();
    const bool pending = !sS.r.decided;
    crack_step_warp<T>(a.p, a.w, a.pitch, a.cut_v, a.hist, sS, +1, true);
    if (a.p.two_tips) crack_step_warp<T>(a.p, a.w, a.pitch, a.cut_v, a.hist, sS, -1, true);
    if (threadIdx.x == 0) {
        if (pending && a.p.mode != CRACK_NONE) sS.hist_n += 1;
        *a.st = sS;
    }
}

template <typename T>
cudaError_t launch_finalize(const FinalizeArgs<T> &a, cudaStream_t s)
{
    finalize_kernel<T><<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------- halo exchange

// Row slabs of a decomposed lattice: after each step, each boundary row of a
// slab is copied into the halo row of its neighbour (CTA q copies pair q,
// 16 bytes per thread per iteration; rows are 128-byte aligned and a whole
// number of 16-byte words long).
__global__ void exchange_kernel(const RowCopy *pairs, int64_t words)
{
    const RowCopy c = pairs[blockIdx.x];
    const uint4 *src = static_cast<const uint4 *>(c.src);
    uint4 *dst = static_cast<uint4 *>(c.dst);
    for (int64_t q = threadIdx.x; q < words; q += blockDim.x) dst[q] = src[q];
}

cudaError_t launch_exchange(const RowCopy *pairs, int n_pairs, int64_t row_bytes, cudaStream_t s)
{
    if (n_pairs <= 0) return cudaSuccess;
    exchange_kernel<<<(unsigned)n_pairs, 256, 0, s>>>(pairs, row_bytes / 16);
    return cudaGetLastError();
}

// ------------------------------------------------------- initial w*(t_0)

struct WstarArgs {
    CrackState *st;
    LoadDesc load[4];
    int32_t edge[4];
    double dt;
};

__global__ void wstar_kernel(const WstarArgs a)
{
    if (threadIdx.x < 4) {
        const int e = threadIdx.x;
        a.st->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], a.st->step, a.dt) : 0.0;
    }
}

cudaError_t launch_wstar(CrackState *st, const LoadDesc *load, const int32_t *edge, double dt, cudaStream_t s)
{
    WstarArgs a;
    a.st = st;
    for (int e = 0; e < 4; ++e) { a.load[e] = load[e]; a.edge[e] = edge[e]; }
    a.dt = dt;
    wstar_kernel<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------- macroscopic rule on the edges
//
// The macroscopic rule (Sec. 3.1) on the free and Dirichlet outer edges, run
// after the step kernel on the fields it wrote.  The boundary system S w_B =
// R couples the boundary points only through interior points that are
// boundary points themselves, in two levels:
//   level 1: a non-corner edge point reads x_I, x_II along its edge's inward
//            normal: bulk sites or crack-face points off the edge columns,
//            all final after the step kernel;
//   level 2: a corner reads two points of the other edge, and a crack-face
//            point on an edge column reads the two edge points above or
//            below it; each such read is a level-1 value that the thread
//            computes itself.
// So one thread per edge site solves its own equation exactly and no thread
// reads a site another thread writes.  Polynomials, with the edge half a
// spacing outside the sites (x_B, x_I, x_II at 1/2, 3/2, 5/2 dh): traction
// free w_B = 1.5 w_I - 0.5 w_II; Dirichlet w_B = 8/15 w* + 2/3 w_I - 1/5 w_II
// with w* at the new time level; a corner follows its Dirichlet edge, else
// the bottom / top one.  wdot_B = (w_B - w_B(t)) / dt, and the pad images
// of the site are refreshed.

template <typename T>
struct EdgeRule {
    const T *wn;          // the new fields
    int64_t pitch;
    int32_t dir[4];       // 1: Dirichlet edge
    T ws[4];              // w* at the new time level
    __device__ __forceinline__ T w(int i, int j) const { return wn[(int64_t)j * pitch + i]; }
    __device__ __forceinline__ T rule(int e, T wI, T wII) const
    {
        if (dir[e])
            return (T)(8.0 / 15.0) * ws[e] + (T)(2.0 / 3.0) * wI - (T)0.2 * wII;
        return (T)1.5 * wI - (T)0.5 * wII;
    }
    // a non-corner point of edge e from its two sites along the inward normal
    __device__ __forceinline__ T point(int e, int i, int j) const
    {
        const int dx = e == LEFT ? 1 : (e == RIGHT ? -1 : 0);
        const int dy = e == BOTTOM ? 1 : (e == TOP ? -1 : 0);
        return rule(e, w(i + dx, j + dy), w(i + 2 * dx, j + 2 * dy));
    }
};

__host__ __device__ __forceinline__ bool ruled(int kind) { return kind == EDGE_FREE || kind == EDGE_DIRICHLET; }

template <typename T, typename D>
__device__ __forceinline__ void edge_rule_at(const StepArgs<T, D> &a, int t)
{
    const int nx = a.nx, ny = a.ny;
    const bool onL = ruled(a.edge[LEFT]), onR = ruled(a.edge[RIGHT]);
    const bool onB = ruled(a.edge[BOTTOM]), onT = ruled(a.edge[TOP]);
    const int nB = onB ? nx : 0, nT = onT ? nx : 0;
    const int jlo = onB ? 1 : 0, jhi = onT ? ny - 2 : ny - 1;
    const int nV = jhi >= jlo ? jhi - jlo + 1 : 0;
    const int nL = onL ? nV : 0, nR = onR ? nV : 0;
    int i, j;
    if (t < nB) { i = t; j = 0; }
    else if ((t -= nB) < nT) { i = t; j = ny - 1; }
    else if ((t -= nT) < nL) { i = 0; j = jlo + t; }
    else if ((t -= nL) < nR) { i = nx - 1; j = jlo + t; }
    else return;

    EdgeRule<T> R;
    R.wn = a.w_out;
    R.pitch = a.pitch;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        R.dir[e] = a.edge[e] == EDGE_DIRICHLET;
        R.ws[e] = (T)a.s_out->wstar[e];
    }
    const int eh = (onL && i == 0) ? LEFT : ((onR && i == nx - 1) ? RIGHT : -1);
    const int ev = (onB && j == 0) ? BOTTOM : ((onT && j == ny - 1) ? TOP : -1);
    const int jc = a.p.jc;
    bool face = false;
    if (a.p.macro && a.p.mode != CRACK_NONE && (j == jc || j == jc - 1)) {
        face = (a.cut_v[(int64_t)(jc - 1) * a.words + (i >> 5)] >> (i & 31)) & 1u;
        if (a.p.q == 9) {
            // D2Q9: also a column of a severed diagonal pair (the crack state
            // of the step, as the update wrote it)
            const int64_t rq = a.s_out->r.tip_q, lq = a.p.two_tips ? a.s_out->l.tip_q : a.p.start_q;
            const int64_t ml = (int64_t)i << kQBits, mr = (int64_t)(i + 1) << kQBits;
            face |= (i >= 1 && lq <= ml && ml <= rq) || (i + 1 <= nx - 1 && lq <= mr && mr <= rq);
        }
    }
    T v;
    if (face) {
        // a crack-face point on an edge column (eh >= 0): its x_I, x_II are
        // the edge points one and two rows further from the crack
        const int s = j == jc ? 1 : -1;
        v = (T)1.5 * R.point(eh, i, j + s) - (T)0.5 * R.point(eh, i, j + 2 * s);
    } else if (eh >= 0 && ev >= 0) {
        const int e = (a.edge[eh] == EDGE_DIRICHLET && a.edge[ev] != EDGE_DIRICHLET) ? eh : ev;
        const int o = e == eh ? ev : eh;
        const int dx = e == LEFT ? 1 : (e == RIGHT ? -1 : 0);
        const int dy = e == BOTTOM ? 1 : (e == TOP ? -1 : 0);
        v = R.rule(e, R.point(o, i + dx, j + dy), R.point(o, i + 2 * dx, j + 2 * dy));
    } else {
        v = R.point(eh >= 0 ? eh : ev, i, j);
    }
    const int64_t P = a.pitch, o = (int64_t)j * P + i;
    const T wd = (v - a.w_in[o]) / a.dt;
    a.w_out[o] = v;
    WdIO<D>::put(a.wd + o, wd, a.wd_scale);
    // pad images of the new value (bounce-back next to a free edge, the
    // wrap-around next to a periodic one)
    T *row = a.w_out + (int64_t)j * P;
    if (i == 0) {
        if (a.edge[LEFT] == EDGE_FREE) row[-1] = v;
        else if (a.edge[LEFT] == EDGE_PERIODIC) row[nx] = v;
    }
    if (i == nx - 1) {
        if (a.edge[RIGHT] == EDGE_FREE) row[nx] = v;
        else if (a.edge[RIGHT] == EDGE_PERIODIC) row[-1] = v;
    }
    if (j == 0) {
        if (a.edge[BOTTOM] == EDGE_FREE) a.w_out[i - P] = v;
        else if (a.edge[BOTTOM] == EDGE_PERIODIC) a.w_out[(int64_t)ny * P + i] = v;
    }
    if (j == ny - 1) {
        if (a.edge[TOP] == EDGE_FREE) a.w_out[(int64_t)ny * P + i] = v;
        else if (a.edge[TOP] == EDGE_PERIODIC) a.w_out[i - P] = v;
    }
    if (!isfinite((double)v) || !isfinite((double)wd)) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
}

template <typename T, typename D>
__global__ void __launch_bounds__(128) edge_rule_kernel(const StepArgs<T, D> a)
{
    pdl_wait();
    pdl_trigger();
    edge_rule_at(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// The same for the lattices of a batch: unit u covers edge sites cb ..
// cb + 127 of lattice inst, whose arguments are read from the descriptor
// table in device memory.
template <typename T, typename D>
__global__ void __launch_bounds__(128) batch_edge_rule_kernel(const StepArgs<T, D> *descs, const BatchUnit *units, int par)
{
    pdl_wait();
    pdl_trigger();
    const BatchUnit u = units[blockIdx.x];
    edge_rule_at(descs[2 * u.inst + par], u.cb + (int)threadIdx.x);
}

template <typename T, typename D>
int edge_rule_sites(const StepArgs<T, D> &a)
{
    const bool onL = ruled(a.edge[LEFT]), onR = ruled(a.edge[RIGHT]);
    const bool onB = ruled(a.edge[BOTTOM]), onT = ruled(a.edge[TOP]);
    const int jlo = onB ? 1 : 0, jhi = onT ? a.ny - 2 : a.ny - 1;
    const int nV = jhi >= jlo ? jhi - jlo + 1 : 0;
    return (onB ? a.nx : 0) + (onT ? a.nx : 0) + (onL ? nV : 0) + (onR ? nV : 0);
}

template <typename T, typename D>
cudaError_t launch_edge_rule(const StepArgs<T, D> &a, cudaStream_t s)
{
    const int n = edge_rule_sites(a);
    if (n == 0) return cudaSuccess;
    return launch_chained(edge_rule_kernel<T, D>, dim3((unsigned)((n + 127) / 128)), dim3(128), 0, s, a.chained != 0, a);
}

template <typename T, typename D>
int edge_rule_count(const StepArgs<T, D> &a)
{
    return edge_rule_sites(a);
}

template <typename T, typename D>
cudaError_t launch_batch_edge_rule(const StepArgs<T, D> *descs, const BatchUnit *units, int n_units, int par,
                                   cudaStream_t s, bool chained)
{
    if (n_units <= 0) return cudaSuccess;
    return launch_chained(batch_edge_rule_kernel<T, D>, dim3((unsigned)n_units), dim3(128), 0, s, chained, descs, units,
                          par);
}

// ------------------------------------------------------ periodic pad images

// Pad images for fields set from outside: the bounce-back image (the edge
// site's own value) next to free edges, the wrap-around value next to
// periodic ones; pads next to Dirichlet edges are not read.
struct PadEdges {
    int32_t e[4];
};

template <typename T>
__global__ void fill_pads_kernel(T *w, int64_t P, int nx, int ny, PadEdges E)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nx) {
        if (E.e[BOTTOM] == EDGE_FREE) w[-P + t] = w[t];
        else if (E.e[BOTTOM] == EDGE_PERIODIC) w[-P + t] = w[(int64_t)(ny - 1) * P + t];
        if (E.e[TOP] == EDGE_FREE) w[(int64_t)ny * P + t] = w[(int64_t)(ny - 1) * P + t];
        else if (E.e[TOP] == EDGE_PERIODIC) w[(int64_t)ny * P + t] = w[t];
    }
    if (t < ny) {
        T *row = w + (int64_t)t * P;
        if (E.e[LEFT] == EDGE_FREE) row[-1] = row[0];
        else if (E.e[LEFT] == EDGE_PERIODIC) row[-1] = row[nx - 1];
        if (E.e[RIGHT] == EDGE_FREE) row[nx] = row[nx - 1];
        else if (E.e[RIGHT] == EDGE_PERIODIC) row[nx] = row[0];
    }
}

template <typename T>
cudaError_t launch_fill_pads(T *w, int64_t pitch, int nx, int ny, const int32_t *edge, cudaStream_t s)
{
    PadEdges E;
    for (int q = 0; q < 4; ++q) E.e[q] = edge[q];
    const int n = nx > ny ? nx : ny;
    fill_pads_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(w, pitch, nx, ny, E);
    return cudaGetLastError();
}

template const void *step_kernel_ptr<double, double>(bool);
template const void *step_kernel_ptr<float, float>(bool);
template const void *step_kernel_ptr<float, __nv_bfloat16>(bool);
template const void *step_kernel_ptr<float, __half>(bool);
template cudaError_t launch_step<double, double>(const StepArgs<double, double> &, int, cudaStream_t, bool);
template cudaError_t launch_step<float, float>(const StepArgs<float, float> &, int, cudaStream_t, bool);
template cudaError_t launch_step<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> &, int, cudaStream_t, bool);
template cudaError_t launch_step<float, __half>(const StepArgs<float, __half> &, int, cudaStream_t, bool);
template cudaError_t launch_step_rec<double>(const StepArgs<double, double> &, const RecArgs &, int, cudaStream_t);
template cudaError_t launch_step_rec<float>(const StepArgs<float, float> &, const RecArgs &, int, cudaStream_t);
template cudaError_t launch_batch_step<double, double>(const StepArgs<double, double> *, const BatchUnit *, int, int, cudaStream_t, int, int, bool);
template cudaError_t launch_batch_step<float, float>(const StepArgs<float, float> *, const BatchUnit *, int, int, cudaStream_t, int, int, bool);
template cudaError_t launch_batch_step<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> *, const BatchUnit *, int, int, cudaStream_t, int, int, bool);
template cudaError_t launch_batch_step<float, __half>(const StepArgs<float, __half> *, const BatchUnit *, int, int, cudaStream_t, int, int, bool);
template cudaError_t launch_batch_persistent<double, double>(const StepArgs<double, double> *, int, const BatchUnit *, int, const BatchUnit *, int, int, int64_t, GridBarrier *, uint32_t *, long long, int, cudaStream_t);
template cudaError_t launch_batch_persistent<float, float>(const StepArgs<float, float> *, int, const BatchUnit *, int, const BatchUnit *, int, int, int64_t, GridBarrier *, uint32_t *, long long, int, cudaStream_t);
template cudaError_t launch_batch_persistent<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> *, int, const BatchUnit *, int, const BatchUnit *, int, int, int64_t, GridBarrier *, uint32_t *, long long, int, cudaStream_t);
template cudaError_t launch_batch_persistent<float, __half>(const StepArgs<float, __half> *, int, const BatchUnit *, int, const BatchUnit *, int, int, int64_t, GridBarrier *, uint32_t *, long long, int, cudaStream_t);
template cudaError_t launch_wd_to_f32<__nv_bfloat16>(const __nv_bfloat16 *, int64_t, int, int, float, float *, cudaStream_t);
template cudaError_t launch_wd_to_f32<__half>(const __half *, int64_t, int, int, float, float *, cudaStream_t);
template cudaError_t launch_wd_from_f32<__nv_bfloat16>(__nv_bfloat16 *, int64_t, int, int, float, const float *, cudaStream_t);
template cudaError_t launch_wd_from_f32<__half>(__half *, int64_t, int, int, float, const float *, cudaStream_t);
template cudaError_t launch_finalize<float>(const FinalizeArgs<float> &, cudaStream_t);
template cudaError_t launch_finalize<double>(const FinalizeArgs<double> &, cudaStream_t);
template int edge_rule_count<double, double>(const StepArgs<double, double> &);
template int edge_rule_count<float, float>(const StepArgs<float, float> &);
template int edge_rule_count<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> &);
template int edge_rule_count<float, __half>(const StepArgs<float, __half> &);
template cudaError_t launch_batch_edge_rule<double, double>(const StepArgs<double, double> *, const BatchUnit *, int, int, cudaStream_t, bool);
template cudaError_t launch_batch_edge_rule<float, float>(const StepArgs<float, float> *, const BatchUnit *, int, int, cudaStream_t, bool);
template cudaError_t launch_batch_edge_rule<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> *, const BatchUnit *, int, int, cudaStream_t, bool);
template cudaError_t launch_batch_edge_rule<float, __half>(const StepArgs<float, __half> *, const BatchUnit *, int, int, cudaStream_t, bool);
template cudaError_t launch_edge_rule<double, double>(const StepArgs<double, double> &, cudaStream_t);
template cudaError_t launch_edge_rule<float, float>(const StepArgs<float, float> &, cudaStream_t);
template cudaError_t launch_edge_rule<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> &, cudaStream_t);
template cudaError_t launch_edge_rule<float, __half>(const StepArgs<float, __half> &, cudaStream_t);
template const void *step_kernel_ptr<float, Lf>(bool);
template cudaError_t launch_step<float, Lf>(const StepArgs<float, Lf> &, int, cudaStream_t, bool);
template cudaError_t launch_batch_step<float, Lf>(const StepArgs<float, Lf> *, const BatchUnit *, int, int, cudaStream_t, int, int, bool);
template cudaError_t launch_batch_persistent<float, Lf>(const StepArgs<float, Lf> *, int, const BatchUnit *, int, const BatchUnit *, int, int, int64_t, GridBarrier *, uint32_t *, long long, int, cudaStream_t);
template int edge_rule_count<float, Lf>(const StepArgs<float, Lf> &);
template cudaError_t launch_batch_edge_rule<float, Lf>(const StepArgs<float, Lf> *, const BatchUnit *, int, int, cudaStream_t, bool);
template cudaError_t launch_edge_rule<float, Lf>(const StepArgs<float, Lf> &, cudaStream_t);
template cudaError_t batch_step_kernel_ptr<double, double>(int, int, const void **);
template cudaError_t batch_step_kernel_ptr<float, float>(int, int, const void **);
template cudaError_t batch_step_kernel_ptr<float, __nv_bfloat16>(int, int, const void **);
template cudaError_t batch_step_kernel_ptr<float, __half>(int, int, const void **);
template cudaError_t batch_step_kernel_ptr<float, Lf>(int, int, const void **);
template cudaError_t batch_piece_kernel_ptr<double, double>(int, int, const void **);
template cudaError_t launch_batch_pieces<double, double>(const StepArgs<double, double> *, const BatchPiece *, const int32_t *, int, int, cudaStream_t, int, int, bool);
template cudaError_t batch_piece_kernel_ptr<float, float>(int, int, const void **);
template cudaError_t launch_batch_pieces<float, float>(const StepArgs<float, float> *, const BatchPiece *, const int32_t *, int, int, cudaStream_t, int, int, bool);
template cudaError_t batch_piece_kernel_ptr<float, __nv_bfloat16>(int, int, const void **);
template cudaError_t launch_batch_pieces<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> *, const BatchPiece *, const int32_t *, int, int, cudaStream_t, int, int, bool);
template cudaError_t batch_piece_kernel_ptr<float, __half>(int, int, const void **);
template cudaError_t launch_batch_pieces<float, __half>(const StepArgs<float, __half> *, const BatchPiece *, const int32_t *, int, int, cudaStream_t, int, int, bool);
template cudaError_t batch_piece_kernel_ptr<float, Lf>(int, int, const void **);
template cudaError_t launch_batch_pieces<float, Lf>(const StepArgs<float, Lf> *, const BatchPiece *, const int32_t *, int, int, cudaStream_t, int, int, bool);
template cudaError_t launch_fill_pads<float>(float *, int64_t, int, int, const int32_t *, cudaStream_t);
template cudaError_t launch_fill_pads<double>(double *, int64_t, int, int, const int32_t *, cudaStream_t);

}  // namespace lbm
