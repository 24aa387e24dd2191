// lbm_d2q9.cu -- the D2Q9 time step (sm_103a).
//
// The paper builds its method on D2Q5 and notes that the crack handling
// carries over to D2Q9 (Sec. 4.1).  With tau = dt the collision sets every
// distribution to its equilibrium, f_eq^a = W_a g w (W = 2/3 on the axes,
// 1/6 on the diagonals: the isotropic nine-point Laplacian, whose axis weight
// plus twice its diagonal weight is 1, so the wave speed stays c_s), and the
// step is the moment update
//     wdot' = wdot + g sum_a W_a (w(x + c_a) - w(x)),    w' = w + dt wdot'.
// A missing link streams back bounce-back (the site's own value: free edge,
// severed crack link) or anti-bounce-back (2 w* - w: Dirichlet edge, with
// w*(t_n)); a periodic edge wraps.  The diagonal links between rows jc-1 and
// jc cross the crack line at x = (i + 1) dh and are severed when that point
// lies on the closed segment between the crack's two ends (the ends only move
// outwards, so the severed set follows from the tips in the state); the
// vertical links come from the cut mask.  A diagonal link that leaves the
// body through one of its corners follows the Dirichlet edge if just one of
// the two edges is Dirichlet, else the bottom / top edge.
//
// The interior marches like the D2Q5 step kernel (16 bytes per site update:
// w and wdot read and written once); the outer-edge warps and the edge and
// crack rows substitute what each missing or severed link streams back.  As
// in the D2Q5 kernel, the crack step of Alg. 1 that follows step k - 1 is
// applied at the start of step k, here by every CTA of the crack rows whose
// columns a new cut can reach (a diagonal cut touches the columns on both
// sides of its crossing): all reach the same decision, one records it.
#include "lbm_crack.cuh"
#include "lbm_internal.cuh"
#include "lbm_rows.cuh"

namespace lbm {


// The value a link streams back when it leaves the body (ox: across the
// left / right edge, oy: across the bottom / top edge; dx, dy its direction):
// anti-bounce-back 2 w* - w on a Dirichlet edge, bounce-back w otherwise; a
// link through a corner follows the Dirichlet edge if just one of the two is
// Dirichlet, else the bottom / top edge.
// Twice the Dirichlet value of each edge, selected without indexing (so that
// it stays in registers).
// The rate and integration of one D2Q9 site, with every rounding fixed:
// wdot' = wdot + (g_a axis + g_d diag) as fma(g_a, axis, g_d diag) and
// w' = fma(dt, wdot', w).  The sum of two products could otherwise be
// contracted into an FMA either way round, and a compiler may choose
// differently in different code paths (the bare, interior and edge-row
// updates); fixed here, every path -- and so every band partition and every
// row-slab split -- gives the same bits.
__device__ __forceinline__ float d9_rate(float wd, float axis, float diag, float ga, float gd)
{
    return __fadd_rn(wd, __fmaf_rn(ga, axis, __fmul_rn(gd, diag)));
}
__device__ __forceinline__ double d9_rate(double wd, double axis, double diag, double ga, double gd)
{
    return __dadd_rn(wd, __fma_rn(ga, axis, __dmul_rn(gd, diag)));
}
__device__ __forceinline__ float d9_integrate(float w, float wd, float dt) { return __fmaf_rn(dt, wd, w); }
__device__ __forceinline__ double d9_integrate(double w, double wd, double dt) { return __fma_rn(dt, wd, w); }

template <typename T>
struct TwoWs {
    T l, r, b, t;
    __device__ __forceinline__ T operator[](int e) const { return e == LEFT ? l : (e == RIGHT ? r : (e == BOTTOM ? b : t)); }
};

template <typename T>
__device__ __forceinline__ T leaving(const int32_t *edge, const TwoWs<T> &two_ws, bool ox, bool oy, int dx, int dy, T w0)
{
    const int ex = dx < 0 ? LEFT : RIGHT, ey = dy < 0 ? BOTTOM : TOP;
    int e = ox ? ex : ey;
    if (ox && oy) e = (edge[ex] == EDGE_DIRICHLET && edge[ey] != EDGE_DIRICHLET) ? ex : ey;
    return edge[e] == EDGE_DIRICHLET ? two_ws[e] - w0 : w0;
}

// One warp's march up rows [j0, j1): a thread owns one 16-byte vector of a
// row, with rows j-1, j, j+1 of w in registers and the east / west
// neighbours of all three rows from the adjacent lanes (lanes 0 and 31 load
// the halo columns), so each w is loaded about once.  Rows beyond a periodic
// edge are loaded from the other side (likewise the halo column of the
// leftmost thread and the column-0 values the thread owning column nx - 1
// needs).  Rows of warps away from the left and right edges (edge_warp
// false) take the bare update unless they are the bottom or top row or a
// crack row; the others substitute the value each missing or severed link
// streams back.
// SPECIAL = false: a warp away from the left and right edges in a band that
// holds no edge row, no crack row and no row beyond a periodic edge (its
// rows are all bare updates): compiled without the periodic remapping, the
// corner column loads and the per-row checks.
template <typename T, bool SPECIAL = true>
__device__ __forceinline__ T march9(const StepArgs<T, T> &a, int x0, int j0, int j1, int64_t lq, int64_t rq,
                                    const TwoWs<T> &two_ws, bool edge_warp)
{
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny, jc = a.p.jc;
    const bool crack = a.p.mode != CRACK_NONE;
    const bool per_x = a.edge[LEFT] == EDGE_PERIODIC, per_y = a.edge[BOTTOM] == EDGE_PERIODIC;
    const bool halo_b = a.edge[BOTTOM] == EDGE_HALO, halo_t = a.edge[TOP] == EDGE_HALO;
    const int kr = nx - 1 - x0;                       // element holding column nx - 1, if in [0, N)
    const bool owns_last = SPECIAL && kr >= 0 && kr < N && per_x;
    const int64_t P = a.pitch;
    const T *wbase = a.w_in;
    const int hl_col = (SPECIAL && x0 == 0 && per_x) ? nx - 1 : x0 - 1;
    const T ga = a.g * (T)(2.0 / 3.0), gd = a.g * (T)(1.0 / 6.0), dt = a.dt;

    // issue the loads of a row: the vector, the halo column of lanes 0 / 31
    // (l, rt) and the east neighbour of column nx - 1 across a periodic edge (z)
    auto load = [&](int r, R &v, T &l, T &rt, T &z) {
        if (SPECIAL && per_y) r = r < 0 ? r + ny : (r >= ny ? r - ny : r);
        const T *row = wbase + (int64_t)r * P;
        ldg_row(row + x0, v);
        l = lane == 0 ? row[hl_col] : (T)0;
        rt = lane == 31 ? row[x0 + N] : (T)0;
        z = owns_last ? row[0] : (T)0;
    };
    // the west / east neighbours of a row's first and last element, once its
    // loads have arrived (one iteration after they were issued)
    auto sides = [&](const R &v, T &l, T &rt) {
        const T su = __shfl_up_sync(kFull, v.v[N - 1], 1), sd = __shfl_down_sync(kFull, v.v[0], 1);
        if (lane != 0) l = su;
        if (lane != 31) rt = sd;
    };
    R wb, wc, wa, wdv;
    T lb, rb, zb, lc, rc, zc, la, ra, za;
    load(j0 - 1, wb, lb, rb, zb);
    load(j0, wc, lc, rc, zc);
    load(j0 + 1, wa, la, ra, za);
    ld_row(a.wd + x0 + (int64_t)j0 * P, wdv);
    sides(wb, lb, rb);
    sides(wc, lc, rc);
    sides(wa, la, ra);
    T acc = (T)0;
    for (int j = j0; j < j1; ++j) {
        R wn, wdn;
        T ln = (T)0, rn = (T)0, zn = (T)0;
        const bool more = j + 1 < j1;
        if (more) {
            load(j + 2, wn, ln, rn, zn);
            ld_row(a.wd + x0 + (int64_t)(j + 1) * P, wdn);
        }
        R wnew, wdnew;
        const bool crow = SPECIAL && crack && (j == jc - 1 || j == jc);
        if (!SPECIAL) {
            // the bare update from the column sums of the rows above and
            // below, s_k = w_a + w_b, each formed once: the axis sum is
            // s_k + (w_W + w_E), the diagonal sum s_{k-1} + s_{k+1} (the
            // general path groups both alike, so that every path, and so
            // every band partition, gives the same bits); each difference
            // with 4 w is taken before the weights, so the rounding stays at
            // the scale of the Laplacians
            T sc[N + 2];
            sc[0] = la + lb;
#pragma unroll
            for (int k = 0; k < N; ++k) sc[k + 1] = wa.v[k] + wb.v[k];
            sc[N + 1] = ra + rb;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const T wl = k == 0 ? lc : wc.v[k - 1], wr = k == N - 1 ? rc : wc.v[k + 1];
                const T axis = (sc[k + 1] + (wl + wr)) - (T)4 * wc.v[k];
                const T diag = (sc[k] + sc[k + 2]) - (T)4 * wc.v[k];
                wdnew.v[k] = d9_rate(wdv.v[k], axis, diag, ga, gd);
                wnew.v[k] = d9_integrate(wc.v[k], wdnew.v[k], dt);
            }
            stg_row(a.w_out + x0 + (int64_t)j * P, wnew);
            stg_row(a.wd + x0 + (int64_t)j * P, wdnew);
            acc += wnew.v[0];
        } else if (!crow && (j != 0 || halo_b) && (j != ny - 1 || halo_t)) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const T wl = k == 0 ? lc : wc.v[k - 1], wr = k == N - 1 ? rc : wc.v[k + 1];
                const T al = k == 0 ? la : wa.v[k - 1], ar = k == N - 1 ? ra : wa.v[k + 1];
                const T bl = k == 0 ? lb : wb.v[k - 1], br = k == N - 1 ? rb : wb.v[k + 1];
                const T axis = ((wa.v[k] + wb.v[k]) + (wl + wr)) - (T)4 * wc.v[k];
                const T diag = ((al + bl) + (ar + br)) - (T)4 * wc.v[k];
                wdnew.v[k] = d9_rate(wdv.v[k], axis, diag, ga, gd);
                wnew.v[k] = d9_integrate(wc.v[k], wdnew.v[k], dt);
            }
            if (!edge_warp) {
                stg_row(a.w_out + x0 + (int64_t)j * P, wnew);
                stg_row(a.wd + x0 + (int64_t)j * P, wdnew);
                acc += wnew.v[0];
            } else {
                // a warp at the left or right edge: redo the edge columns with
                // the values their links across the edge stream back
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const int i = x0 + k;
                    if (!((i == 0 && !per_x) || i == nx - 1)) continue;
                    const T w0 = wc.v[k];
                    T wl = k == 0 ? lc : wc.v[k - 1], wr = k == N - 1 ? rc : wc.v[k + 1];
                    T al = k == 0 ? la : wa.v[k - 1], ar = k == N - 1 ? ra : wa.v[k + 1];
                    T bl = k == 0 ? lb : wb.v[k - 1], br = k == N - 1 ? rb : wb.v[k + 1];
                    if (i == nx - 1) {
                        if (per_x) { wr = zc; ar = za; br = zb; }
                        else {
                            wr = leaving(a.edge, two_ws, true, false, 1, 0, w0);
                            ar = leaving(a.edge, two_ws, true, false, 1, 1, w0);
                            br = leaving(a.edge, two_ws, true, false, 1, -1, w0);
                        }
                    }
                    if (i == 0 && !per_x) {
                        wl = leaving(a.edge, two_ws, true, false, -1, 0, w0);
                        al = leaving(a.edge, two_ws, true, false, -1, 1, w0);
                        bl = leaving(a.edge, two_ws, true, false, -1, -1, w0);
                    }
                    const T axis = ((wa.v[k] + wb.v[k]) + (wl + wr)) - (T)4 * w0;
                    const T diag = ((al + bl) + (ar + br)) - (T)4 * w0;
                    wdnew.v[k] = d9_rate(wdv.v[k], axis, diag, ga, gd);
                    wnew.v[k] = d9_integrate(w0, wdnew.v[k], dt);
                }
                if (x0 + N <= nx) {
                    stg_row(a.w_out + x0 + (int64_t)j * P, wnew);
                    stg_row(a.wd + x0 + (int64_t)j * P, wdnew);
                } else {
#pragma unroll
                    for (int k = 0; k < N; ++k)
                        if (x0 + k < nx) {
                            a.w_out[x0 + k + (int64_t)j * P] = wnew.v[k];
                            a.wd[x0 + k + (int64_t)j * P] = wdnew.v[k];
                        }
                }
                if (x0 < nx) acc += wnew.v[0];
            }
        } else {
            uint32_t vbits = 0;
            if (crow && x0 < nx) vbits = a.cut_v[(int64_t)(jc - 1) * a.words + (x0 >> 5)] >> (x0 & 31);
            const bool below = j == jc - 1;           // crack row under the crack line: its links go up
            // a row slab's halo edge is no edge: the row beyond it is the
            // neighbouring slab's, loaded like any other row
            const bool bot = j == 0 && !per_y && !halo_b, top = j == ny - 1 && !per_y && !halo_t;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int i = x0 + k;
                const T w0 = wc.v[k];
                const bool lft = i == 0 && !per_x, rgt = i == nx - 1 && !per_x;
                const bool wrapr = i == nx - 1 && per_x;
                T wl = k == 0 ? lc : wc.v[k - 1], wr = k == N - 1 ? rc : wc.v[k + 1];
                T al = k == 0 ? la : wa.v[k - 1], ar = k == N - 1 ? ra : wa.v[k + 1];
                T bl = k == 0 ? lb : wb.v[k - 1], br = k == N - 1 ? rb : wb.v[k + 1];
                T up = wa.v[k], dn = wb.v[k];
                if (wrapr) { wr = zc; ar = za; br = zb; }
                // the links across the crack line
                bool cv = false, cl = false, cr = false;
                if (crow) {
                    cv = (vbits >> k) & 1u;
                    const int64_t ml = (int64_t)i << kQBits, mr = (int64_t)(i + 1) << kQBits;
                    cl = i >= 1 && lq <= ml && ml <= rq;
                    cr = i + 1 <= nx - 1 && lq <= mr && mr <= rq;
                }
                // west, east, north, south
                if (lft) wl = leaving(a.edge, two_ws, true, false, -1, 0, w0);
                if (rgt) wr = leaving(a.edge, two_ws, true, false, 1, 0, w0);
                if (top) up = leaving(a.edge, two_ws, false, true, 0, 1, w0);
                else if (crow && below && cv) up = w0;
                if (bot) dn = leaving(a.edge, two_ws, false, true, 0, -1, w0);
                else if (crow && !below && cv) dn = w0;
                // the diagonals
                if (crow && below && cl) al = w0;
                else if (lft || top) al = leaving(a.edge, two_ws, lft, top, -1, 1, w0);
                if (crow && below && cr) ar = w0;
                else if (rgt || top) ar = leaving(a.edge, two_ws, rgt, top, 1, 1, w0);
                if (crow && !below && cl) bl = w0;
                else if (lft || bot) bl = leaving(a.edge, two_ws, lft, bot, -1, -1, w0);
                if (crow && !below && cr) br = w0;
                else if (rgt || bot) br = leaving(a.edge, two_ws, rgt, bot, 1, -1, w0);
                const T axis = ((up + dn) + (wl + wr)) - (T)4 * w0;
                const T diag = ((al + bl) + (ar + br)) - (T)4 * w0;
                wdnew.v[k] = d9_rate(wdv.v[k], axis, diag, ga, gd);
                wnew.v[k] = d9_integrate(w0, wdnew.v[k], dt);
            }
            if (x0 + N <= nx) {
                stg_row(a.w_out + x0 + (int64_t)j * P, wnew);
                stg_row(a.wd + x0 + (int64_t)j * P, wdnew);
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k)
                    if (x0 + k < nx) {
                        a.w_out[x0 + k + (int64_t)j * P] = wnew.v[k];
                        a.wd[x0 + k + (int64_t)j * P] = wdnew.v[k];
                    }
            }
            if (x0 < nx) acc += wnew.v[0];
        }
        wb = wc; lb = lc; rb = rc; zb = zc;
        wc = wa; lc = la; rc = ra; zc = za;
        if (more) {
            sides(wn, ln, rn);
            wa = wn; la = ln; ra = rn; za = zn;
            wdv = wdn;
        }
    }
    return acc;
}

// The grid is (column blocks of kThreads vectors) x (the handle's bands: as
// for the D2Q5 step, the crack rows jc - 1 and jc lie in sub-bands of their
// own, one or three rows tall, so that the CTAs that run the pending crack
// step first have few rows after it, and the other bands are as tall as one
// wave of resident CTAs allows).
// One CTA of the D2Q9 step: column block cb of band `band` of the lattice
// that `a` describes (the kernel parameter block, or a copy in shared memory).
template <typename T>
__device__ __forceinline__ void d2q9_cta(const StepArgs<T, T> &a, int cb, int band, CrackState &sS)
{
    constexpr int N = Vec<T>::N;
    constexpr int cols = kThreads * N;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nx = a.nx, ny = a.ny, jc = a.p.jc;
    const int x0 = (cb * kThreads + tid) * N;
    const int xw0 = (cb * kThreads + (tid & ~31)) * N;
    const Unit U = a.units[band];
    const int j0 = U.j0, j1 = U.j1;
    const bool crack = a.p.mode != CRACK_NONE;
    const bool edge_warp = xw0 == 0 || xw0 + 32 * N - 1 >= nx - 1;
    const CrackParams &p = a.p;
    const CrackState *s_in = a.s_in;
    int64_t lq = 0, rq = -1;
    if (crack) {
        // the CTAs of the crack rows near each end's next vertical link run
        // its pending crack step: i_next for the right end, i_prev for the
        // left one; the diagonal crossings a step can add lie between columns
        // i_next - 1 and i_next + 2 (i_prev - 2 and i_prev + 1)
        const bool crack_rows = (jc - 1 >= j0 && jc - 1 < j1) || (jc >= j0 && jc < j1);
        const bool commit_band = jc - 1 >= j0 && jc - 1 < j1;
        const int c0 = cb * cols, c1 = c0 + cols - 1;
        int i_next = max(s_in->i_last + 1, s_in->i_first);
        i_next = min(max(i_next, 0), nx - 1);
        int i_prev = min(s_in->i_first - 1, s_in->i_last);
        i_prev = min(max(i_prev, 0), nx - 1);
        const bool right_here = crack_rows && c0 <= i_next + 2 && c1 >= i_next - 1;
        const bool left_here = crack_rows && p.two_tips && c0 <= i_prev + 1 && c1 >= i_prev - 2;
        if (right_here || left_here) {
            const bool commit_r = right_here && commit_band && cb == i_next / cols;
            const bool commit_l = left_here && commit_band && cb == i_prev / cols;
            if (tid < 32) {
                if (tid == 0) sS = *s_in;
                __syncwarp();
                const bool pending = !sS.r.decided;   // not yet applied by a deferred crack step
                if (right_here) crack_step_warp<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, +1, commit_r);
                if (left_here) crack_step_warp<T>(p, a.w_in, a.pitch, a.cut_v, a.hist, sS, -1, commit_l);
                if (tid == 0 && commit_r) {
                    CrackState *o = a.s_out;
                    const int64_t n = sS.step + 1;
                    o->step = n;
                    o->hist_n = sS.hist_n + (pending ? 1 : 0);
                    o->i_last = sS.i_last;
                    if (!p.two_tips) o->i_first = sS.i_first;
                    o->r = sS.r;
                    o->r.decided = 0;
                    for (int e = 0; e < 4; ++e)
                        o->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)p.dt) : 0.0;
                }
                if (tid == 0 && commit_l) {
                    CrackState *o = a.s_out;
                    o->i_first = sS.i_first;
                    o->l = sS.l;
                    o->l.decided = 0;
                }
            }
            __syncthreads();   // this CTA's new cuts and tips, for all of its threads
            rq = sS.r.tip_q;
            lq = p.two_tips ? sS.l.tip_q : p.start_q;
        } else {
            rq = s_in->r.tip_q;
            lq = p.two_tips ? s_in->l.tip_q : p.start_q;
        }
    } else if (cb == 0 && band == 0 && tid == 0) {
        // no crack: only the step counter and the Dirichlet values advance
        CrackState st = *s_in;
        const int64_t n = st.step + 1;
        st.step = n;
        st.r.decided = 1;
        st.l.decided = 1;
        for (int e = 0; e < 4; ++e)
            st.wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)p.dt) : 0.0;
        *a.s_out = st;
    }
    const TwoWs<T> two_ws{(T)2 * (T)a.s_in->wstar[LEFT], (T)2 * (T)a.s_in->wstar[RIGHT],
                          (T)2 * (T)a.s_in->wstar[BOTTOM], (T)2 * (T)a.s_in->wstar[TOP]};
    // warps wholly right of the lattice have nothing to load or store; a warp
    // away from the left / right edges in a band of bare rows takes the
    // march compiled without the edge and crack handling
    const bool per_y = a.edge[BOTTOM] == EDGE_PERIODIC;
    // (the rows next to a row slab's halo edge are bare rows too)
    const bool bare_band = (j0 > 0 || a.edge[BOTTOM] == EDGE_HALO) && (j1 < ny || a.edge[TOP] == EDGE_HALO) &&
                           !(crack && j0 <= jc && j1 >= jc - 1) && !per_y;
    T acc = (T)0;
    if (xw0 < nx) {
        if (!edge_warp && bare_band) acc = march9<T, false>(a, x0, j0, j1, lq, rq, two_ws, false);
        else acc = march9<T, true>(a, x0, j0, j1, lq, rq, two_ws, edge_warp);
    }
    // a non-finite w (or wdot, which enters w) turns the sum of the first
    // element of each vector non-finite within a step or two
    if (__any_sync(0xffffffffu, !isfinite(acc)) && lane == 0) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2)
    d2q9_step_kernel(const StepArgs<T, T> a)
{
    __shared__ CrackState sS;
    pdl_wait();
    pdl_trigger();
    d2q9_cta<T>(a, blockIdx.x, blockIdx.y, sS);
}

// Many D2Q9 lattices in one launch: CTA u runs unit u of the batch (column
// block cb of band `band` of lattice inst) with its lattice's arguments for
// the current parity copied to shared memory first; the per-CTA code is the
// single-lattice kernel's, so each lattice ends bit-identical to its solo run.
template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2)
    batch_d2q9_kernel(const StepArgs<T, T> *descs, const BatchUnit *units, int par)
{
    __shared__ CrackState sS;
    __shared__ __align__(16) StepArgs<T, T> sa;
    pdl_wait();
    pdl_trigger();
    const BatchUnit u = units[blockIdx.x];
    const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + 2 * u.inst + par);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
    for (int q = threadIdx.x; q < (int)(sizeof(StepArgs<T, T>) / 4); q += kThreads) dst[q] = src[q];
    __syncthreads();
    d2q9_cta<T>(sa, u.cb, u.band, sS);
}

template <typename T>
cudaError_t launch_d2q9_step(const StepArgs<T, T> &a, cudaStream_t s)
{
    const dim3 grid((unsigned)a.ncb, (unsigned)a.n_bands);
    return launch_chained(d2q9_step_kernel<T>, grid, dim3(kThreads), 0, s, a.chained != 0, a);
}

// The macroscopic rule on the D2Q9 crack faces (Sec. 3.1), after the update:
// a site of rows jc - 1 and jc is a boundary point when its column has a
// severed vertical link or is one of the two columns of a severed diagonal
// pair; it takes the normal of the crack face its link crosses, so x_I, x_II
// are the next two sites of its column away from the crack:
// w_B = 1.5 w_I - 0.5 w_II, wdot_B = (w_B - w_B(t)) / dt.  The crack state of
// the step (the cuts in force during it) is the one the update wrote to
// s_out.  One thread per column; x_I, x_II are never boundary points.
template <typename T>
__device__ __forceinline__ void d2q9_face_at(const StepArgs<T, T> &a, int i)
{
    if (i >= a.nx) return;
    const int nx = a.nx, jc = a.p.jc;
    const CrackState *st = a.s_out;
    const int64_t rq = st->r.tip_q, lq = a.p.two_tips ? st->l.tip_q : a.p.start_q;
    const int64_t ml = (int64_t)i << kQBits, mr = (int64_t)(i + 1) << kQBits;
    const bool vcut = (a.cut_v[(int64_t)(jc - 1) * a.words + (i >> 5)] >> (i & 31)) & 1u;
    const bool dl = i >= 1 && lq <= ml && ml <= rq, dr = i + 1 <= nx - 1 && lq <= mr && mr <= rq;
    if (!(vcut || dl || dr)) return;
    const int64_t P = a.pitch;
    const T *wn = a.w_out;
    const T inv_dt = (T)1 / a.dt;
    const T up = (T)1.5 * wn[(int64_t)(jc + 1) * P + i] - (T)0.5 * wn[(int64_t)(jc + 2) * P + i];
    const T dn = (T)1.5 * wn[(int64_t)(jc - 2) * P + i] - (T)0.5 * wn[(int64_t)(jc - 3) * P + i];
    const int64_t ou = (int64_t)jc * P + i, od = (int64_t)(jc - 1) * P + i;
    const T wdu = (up - a.w_in[ou]) * inv_dt, wdd = (dn - a.w_in[od]) * inv_dt;
    a.w_out[ou] = up;
    a.wd[ou] = wdu;
    a.w_out[od] = dn;
    a.wd[od] = wdd;
    if (!isfinite(up) || !isfinite(dn)) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
}

template <typename T>
__global__ void __launch_bounds__(128) d2q9_face_kernel(const StepArgs<T, T> a)
{
    pdl_wait();
    pdl_trigger();
    d2q9_face_at(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// The face rule of many D2Q9 lattices in one launch: unit u covers columns
// u.cb .. u.cb + 127 of lattice u.inst.
template <typename T>
__global__ void __launch_bounds__(128) batch_d2q9_face_kernel(const StepArgs<T, T> *descs, const BatchUnit *units, int par)
{
    pdl_wait();
    pdl_trigger();
    const BatchUnit u = units[blockIdx.x];
    d2q9_face_at(descs[2 * u.inst + par], u.cb + (int)threadIdx.x);
}

template <typename T>
cudaError_t launch_d2q9_faces(const StepArgs<T, T> &a, cudaStream_t s)
{
    return launch_chained(d2q9_face_kernel<T>, dim3((unsigned)((a.nx + 127) / 128)), dim3(128), 0, s, a.chained != 0,
                          a);
}

template <typename T>
cudaError_t launch_batch_d2q9(const StepArgs<T, T> *descs, const BatchUnit *units, int n_units, const BatchUnit *funits,
                             int n_funits, int par, cudaStream_t s, bool chained)
{
    cudaError_t e = cudaSuccess;
    if (n_units > 0)
        e = launch_chained(batch_d2q9_kernel<T>, dim3((unsigned)n_units), dim3(kThreads), 0, s, chained, descs, units,
                           par);
    if (e == cudaSuccess && n_funits > 0)
        e = launch_chained(batch_d2q9_face_kernel<T>, dim3((unsigned)n_funits), dim3(128), 0, s, chained, descs, funits,
                           par);
    return e;
}

template cudaError_t launch_batch_d2q9<double>(const StepArgs<double, double> *, const BatchUnit *, int,
                                               const BatchUnit *, int, int, cudaStream_t, bool);
template cudaError_t launch_batch_d2q9<float>(const StepArgs<float, float> *, const BatchUnit *, int,
                                              const BatchUnit *, int, int, cudaStream_t, bool);
template cudaError_t launch_d2q9_faces<double>(const StepArgs<double, double> &, cudaStream_t);
template cudaError_t launch_d2q9_faces<float>(const StepArgs<float, float> &, cudaStream_t);
template cudaError_t launch_d2q9_step<double>(const StepArgs<double, double> &, cudaStream_t);
template cudaError_t launch_d2q9_step<float>(const StepArgs<float, float> &, cudaStream_t);

}  // namespace lbm
