// lbm_line.cu -- the time step of a lattice with a straight crack in any
// direction (sm_103a).
//
// Sec. 4.1 models the crack as a line independent of the lattice that grows
// along a given direction; aligning the lattice with it is a convenience.
// Here the crack runs from its start through its tip along the unit
// direction c.  The tip lives on the 2^-32 dh grid; an advance Delta a c is
// rounded per component, and the step severs every link (H or V) that the
// segment from the old to the new tip intersects (closed segments, exact
// integer orientation tests), so the crack is the polyline of its tips.  A
// tip that meets the body's boundary stops there.  The faces are link-local
// (bounce-back).  K (eq. sif) is the least-squares fit over the severed
// links whose midpoint m lies at r = (x_tip - m) . c in [r_min, r_min + W)
// behind the tip, with the opening delta = w(left of c) - w(right of c) of
// the link's two sites; r is formed without fused multiply-adds, so the
// window holds the same pairs as in any other implementation of this
// reading.
//
// The update is the D2Q5 moment form with bounce-back on every severed
// link, marched up the rows like the step kernel (16 bytes per site update),
// reading the cut words of the rows the crack can reach.  As in the step
// kernel, the crack step that follows step k - 1 is applied at the start of
// step k, here by every CTA with sites within two spacings of the tip (the
// links an advance of less than one spacing severs have both ends there):
// all reach the same decision and set the same bits -- the new links lie
// less than half a spacing behind the old tip, while the K window starts
// more than half a spacing behind it, so no CTA's K sees another's new cuts
// -- and the CTA holding the tip's cell records it.
#include "lbm_crack.cuh"
#include "lbm_internal.cuh"
#include "lbm_rows.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ int64_t lo64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t hi64(int64_t a, int64_t b) { return a < b ? b : a; }

__device__ __forceinline__ int64_t centre_q(int i) { return (int64_t)(2 * i + 1) << (kQBits - 1); }

__device__ __forceinline__ int64_t floor_div_q(int64_t a) { return a >= 0 ? a >> kQBits : -((-a + ((int64_t)1 << kQBits) - 1) >> kQBits); }

// Sign of the cross product (b - a) x (c - a), exact.
__device__ __forceinline__ int orient_q(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy)
{
    const __int128 v = (__int128)(bx - ax) * (__int128)(cy - ay) - (__int128)(by - ay) * (__int128)(cx - ax);
    return (v > 0) - (v < 0);
}

__device__ __forceinline__ bool within(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py)
{
    return px >= lo64(ax, bx) && px <= hi64(ax, bx) && py >= lo64(ay, by) && py <= hi64(ay, by);
}

// Do the closed segments p1p2 and q1q2 meet?  (Proper crossing, or an end
// point of one on the other.)
__device__ bool segments_meet(int64_t p1x, int64_t p1y, int64_t p2x, int64_t p2y, int64_t q1x, int64_t q1y,
                              int64_t q2x, int64_t q2y)
{
    const int a = orient_q(q1x, q1y, q2x, q2y, p1x, p1y), b = orient_q(q1x, q1y, q2x, q2y, p2x, p2y);
    const int c = orient_q(p1x, p1y, p2x, p2y, q1x, q1y), d = orient_q(p1x, p1y, p2x, p2y, q2x, q2y);
    if (a * b < 0 && c * d < 0) return true;
    return (a == 0 && within(q1x, q1y, q2x, q2y, p1x, p1y)) || (b == 0 && within(q1x, q1y, q2x, q2y, p2x, p2y)) ||
           (c == 0 && within(p1x, p1y, p2x, p2y, q1x, q1y)) || (d == 0 && within(p1x, p1y, p2x, p2y, q2x, q2y));
}

// A tip moving from (px, py) to (qx, qy) that reaches or crosses the body's
// boundary [0, nx] x [0, ny] (grid units) stops where the segment meets it
// first, in exact integer arithmetic (quotients truncated towards zero).
// Returns true if it stopped.
__device__ bool line_clamp(const CrackParams &p, int64_t px, int64_t py, int64_t &qx, int64_t &qy)
{
    const int64_t X = p.clamp_q, Y = p.clamp_yq;
    const int64_t dx = qx - px, dy = qy - py;
    const bool hx = (dx > 0 && qx >= X) || (dx < 0 && qx <= 0);
    const bool hy = (dy > 0 && qy >= Y) || (dy < 0 && qy <= 0);
    if (!hx && !hy) return false;
    const int64_t fx = dx > 0 ? X : 0, fy = dy > 0 ? Y : 0;
    const __int128 ux = (__int128)(fx - px), uy = (__int128)(fy - py);
    bool xfirst = hx;
    if (hx && hy) {
        const __int128 ax = ux < 0 ? -ux : ux, ay = uy < 0 ? -uy : uy;
        const __int128 adx = dx < 0 ? -(__int128)dx : (__int128)dx, ady = dy < 0 ? -(__int128)dy : (__int128)dy;
        xfirst = ax * ady <= ay * adx;
    }
    if (xfirst) {
        qx = fx;
        qy = py + (int64_t)(ux * (__int128)dy / (__int128)dx);
    } else {
        qy = fy;
        qx = px + (int64_t)(uy * (__int128)dx / (__int128)dy);
    }
    return true;
}

struct LineSums {
    double num, den, r_min;
    int np;
};

// Step (1) of the crack step: the least-squares sums of eq. sif over the
// severed links in the window, by one warp (every lane gets the sums).  The
// candidates are the sites around the window's stretch of the crack,
// widened by two spacings (a severed link's ends lie within 1.3 spacings of
// the crack line).
template <typename T>
__device__ LineSums line_eval_warp(const CrackParams &p, const T *w, int64_t P, const uint32_t *cut_h,
                                   const uint32_t *cut_v, const TipState &E)
{
    const int lane = threadIdx.x & 31;
    const double r_min = p.r_min_fixed > 0.0 ? p.r_min_fixed : p.r0 / (1.0 - E.v_prev);   // eq. r(v)
    const double lo = r_min / p.dh, hi = (r_min + p.fit_width) / p.dh;
    const double tx = (double)E.tip_q * kTwoM32, ty = (double)E.tip_yq * kTwoM32;
    const double ax = tx - lo * p.dir_x, bx = tx - hi * p.dir_x, ay = ty - lo * p.dir_y, by = ty - hi * p.dir_y;
    const double X = (double)p.nx, Y = (double)p.ny;
    auto cl = [](double v, double lim) { return fmin(fmax(v, -4.0), lim + 4.0); };
    int i0 = (int)floor(cl(fmin(ax, bx), X) - 2.0), i1 = (int)ceil(cl(fmax(ax, bx), X) + 2.0);
    int j0 = (int)floor(cl(fmin(ay, by), Y) - 2.0), j1 = (int)ceil(cl(fmax(ay, by), Y) + 2.0);
    i0 = max(i0, 0);
    j0 = max(j0, 0);
    i1 = min(i1, p.nx - 1);
    j1 = min(j1, p.ny - 1);
    const int ni = i1 - i0 + 1, nj = j1 - j0 + 1;
    const int total = (ni > 0 && nj > 0) ? ni * nj : 0;
    const bool k1_left_v = p.dir_x > 0.0, k1_left_h = p.dir_y < 0.0;
    double num = 0.0, den = 0.0;
    int np = 0;
    for (int q = lane; q < total; q += 32) {
        const int i = i0 + q % ni, j = j0 + q / ni;
#pragma unroll
        for (int vert = 0; vert < 2; ++vert) {
            bool cut;
            int64_t mx, my;
            if (!vert) {
                if (i + 1 >= p.nx) continue;
                cut = (__ldcg(cut_h + (int64_t)j * p.words + (i >> 5)) >> (i & 31)) & 1u;
                mx = (int64_t)(i + 1) << kQBits;
                my = centre_q(j);
            } else {
                if (j + 1 >= p.ny) continue;
                cut = (__ldcg(cut_v + (int64_t)j * p.words + (i >> 5)) >> (i & 31)) & 1u;
                mx = centre_q(i);
                my = (int64_t)(j + 1) << kQBits;
            }
            if (!cut) continue;
            const double px = __dmul_rn((double)(E.tip_q - mx) * kTwoM32, p.dir_x);
            const double py = __dmul_rn((double)(E.tip_yq - my) * kTwoM32, p.dir_y);
            const double r_h = __dadd_rn(px, py);
            if (!(r_h >= lo && r_h < hi)) continue;
            const double w0 = (double)w[(int64_t)j * P + i];
            const double w1 = (double)(vert ? w[(int64_t)(j + 1) * P + i] : w[(int64_t)j * P + i + 1]);
            const double delta = (vert ? k1_left_v : k1_left_h) ? w1 - w0 : w0 - w1;
            const double r = r_h * p.dh;
            const double sf = sqrt(r / (2.0 * kPi));
            num += delta * sf;
            den += sf * sf;
            ++np;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
        np += __shfl_xor_sync(0xffffffffu, np, o);
    }
    return LineSums{num, den, r_min, np};
}

// The crack step of Alg. 1 for a crack in any direction, by one warp on the
// state S (shared memory): K, the criterion, the advance (with the stop at
// the boundary), the severed links, the tip's fields of S and, if `commit`,
// the history record at hist_n (tip x in tip, tip y in tipl).
template <typename T>
__device__ void line_step_warp(const CrackParams &p, const T *w, int64_t P, uint32_t *cut_h, uint32_t *cut_v,
                               const History &hist, CrackState &S, bool commit)
{
    const int lane = threadIdx.x & 31;
    TipState &E = S.r;
    if (p.mode == CRACK_NONE || E.decided) {
        __syncwarp();
        if (lane == 0) E.decided = 1;
        __syncwarp();
        return;
    }
    const LineSums c = line_eval_warp<T>(p, w, P, cut_h, cut_v, E);
    // (2) the criterion and (3) the advance: the same scalars on every lane
    const double K = c.np > 0 ? p.mu / 4.0 * c.num / c.den : 0.0;
    int propagate = 0;
    double v = 0.0;
    if (p.mode == CRACK_PRESCRIBED) {
        propagate = 1;
        v = p.v_rel;
    } else if (p.mode == CRACK_KCRIT && c.np > 0 && fabs(K) > p.K_C) {
        const double ratio = fabs(K) / p.K_C;
        propagate = 1;
        v = p.v_max * tanh(sqrt(ratio * ratio * ratio * ratio - 1.0));   // eq. v-tanh
    }
    int32_t flags = E.flags;
    if (!isfinite(K)) flags |= FLAG_NONFINITE;
    int32_t arrested = E.arrested;
    if (arrested) { propagate = 0; v = 0.0; }
    const int64_t px = E.tip_q, py = E.tip_yq;
    int64_t qx = px, qy = py;
    if (propagate) {
        const double adot = v * p.cs;
        const double q = adot * p.dt / p.dh * 4294967296.0;   // Delta a = adot dt, in grid units
        qx = px + __double2ll_rn(q * p.dir_x);
        qy = py + __double2ll_rn(q * p.dir_y);
        if (line_clamp(p, px, py, qx, qy)) { arrested = 1; flags |= FLAG_CLAMPED; }
    }
    const int grew = (qx != px || qy != py) ? 1 : 0;
    if (grew) {
        // (4) sever every link the segment (px, py)-(qx, qy) meets: both ends
        // of such a link lie within one spacing of the segment
        const int64_t one = (int64_t)1 << kQBits, half = one >> 1;
        const int i0 = (int)hi64(0, floor_div_q(lo64(px, qx) - 3 * half));
        const int i1 = (int)lo64(p.nx - 1, floor_div_q(hi64(px, qx) + half) + 1);
        const int j0 = (int)hi64(0, floor_div_q(lo64(py, qy) - 3 * half));
        const int j1 = (int)lo64(p.ny - 1, floor_div_q(hi64(py, qy) + half) + 1);
        const int ni = i1 - i0 + 1, nj = j1 - j0 + 1;
        const int total = (ni > 0 && nj > 0) ? ni * nj : 0;
        for (int t = lane; t < total; t += 32) {
            const int i = i0 + t % ni, j = j0 + t / ni;
            const int64_t cx = centre_q(i), cy = centre_q(j);
            if (i + 1 < p.nx && segments_meet(cx, cy, centre_q(i + 1), cy, px, py, qx, qy))
                atomicOr(&cut_h[(int64_t)j * p.words + (i >> 5)], 1u << (i & 31));
            if (j + 1 < p.ny && segments_meet(cx, cy, cx, centre_q(j + 1), px, py, qx, qy))
                atomicOr(&cut_v[(int64_t)j * p.words + (i >> 5)], 1u << (i & 31));
        }
    }
    __syncwarp();
    if (lane == 0) {
        E.tip_q = qx;
        E.tip_yq = qy;
        E.v_prev = p.mode == CRACK_PRESCRIBED ? p.v_rel : v;
        E.K = K;
        E.v = v;
        E.r_min = c.r_min;
        E.npairs = c.np;
        E.grew = grew;
        E.flags = flags;
        E.arrested = arrested;
        if (commit && p.hist_cap > 0) {
            const int64_t h = S.hist_n % p.hist_cap;
            hist.K[h] = K;
            hist.v[h] = v;
            hist.tip[h] = qx;
            hist.tipl[h] = qy;
            hist.np[h] = c.np;
        }
        E.decided = 1;
    }
    __syncwarp();
}

// One warp's march up rows [j0, j1): a thread owns one 16-byte vector of a
// row, with rows j-1, j, j+1 of w in registers and the east / west
// neighbours of the centre row from the adjacent lanes (lanes 0 and 31 load
// the halo columns).  Free and periodic edges come in through the pads,
// Dirichlet edges by anti-bounce-back; a severed link (of the rows the crack
// can reach) streams back the site's own value.
template <typename T>
__device__ __forceinline__ T line_march(const StepArgs<T, T> &a, const EdgeValues<T> &E, int x0, int j0, int j1)
{
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const uint32_t kMask = (1u << N) - 1u;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny;
    const int64_t P = a.pitch;
    const T *wb = a.w_in;
    const int rlo = a.p.row_lo, rhi = a.p.row_hi;
    const bool own = x0 < nx;
    auto load = [&](int r, R &v, T &l, T &rt) {
        const T *row = wb + (int64_t)r * P;
        ldg_row(row + x0, v);
        l = lane == 0 ? row[x0 - 1] : (T)0;
        rt = lane == 31 ? row[x0 + N] : (T)0;
    };
    auto sides = [&](const R &v, T &l, T &rt) {
        const T su = __shfl_up_sync(kFull, v.v[N - 1], 1), sd = __shfl_down_sync(kFull, v.v[0], 1);
        if (lane != 0) l = su;
        if (lane != 31) rt = sd;
    };
    const bool dir_l = a.edge[LEFT] == EDGE_DIRICHLET, dir_r = a.edge[RIGHT] == EDGE_DIRICHLET;
    R dn, c, up, wdv;
    T lc, rc, lu, ru, l_, r_;
    load(j0 - 1, dn, l_, r_);
    load(j0, c, lc, rc);
    load(j0 + 1, up, lu, ru);
    ld_row(a.wd + x0 + (int64_t)j0 * P, wdv);
    sides(c, lc, rc);
    sides(up, lu, ru);
    T acc = (T)0;
    for (int j = j0; j < j1; ++j) {
        R nxt, wdn;
        T ln = (T)0, rn = (T)0;
        const bool more = j + 1 < j1;
        if (more) {
            load(j + 2, nxt, ln, rn);
            ld_row(a.wd + x0 + (int64_t)(j + 1) * P, wdn);
        }
        // severed links of this row's sites: to the east (cr), west (cl),
        // north (cu) and south (cd)
        uint32_t cr = 0u, cl = 0u, cu = 0u, cd = 0u;
        if (j >= rlo && j <= rhi) {
            const int64_t wo = (int64_t)(x0 >> 5);
            const int sh = x0 & 31;
            if (own) {
                cr = (__ldcg(a.cut_h + (int64_t)j * a.words + wo) >> sh) & kMask;
                if (j + 1 < ny) cu = (__ldcg(a.cut_v + (int64_t)j * a.words + wo) >> sh) & kMask;
                if (j >= 1) cd = (__ldcg(a.cut_v + (int64_t)(j - 1) * a.words + wo) >> sh) & kMask;
            }
            uint32_t lb = (__shfl_up_sync(kFull, cr, 1) >> (N - 1)) & 1u;
            if (lane == 0)
                lb = (x0 >= 1 && x0 - 1 < nx) ? (__ldcg(a.cut_h + (int64_t)j * a.words + ((x0 - 1) >> 5)) >> ((x0 - 1) & 31)) & 1u
                                              : 0u;
            cl = ((cr << 1) | lb) & kMask;
        }
        const bool dir_t = j == ny - 1 && a.edge[TOP] == EDGE_DIRICHLET;
        const bool dir_b = j == 0 && a.edge[BOTTOM] == EDGE_DIRICHLET;
        R wn, wdnew;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T w0 = c.v[k];
            T wl = k == 0 ? lc : c.v[k - 1], wr = k == N - 1 ? rc : c.v[k + 1];
            T u = up.v[k], d = dn.v[k];
            if (dir_t) u = E.two_ws[TOP] - w0;
            else if ((cu >> k) & 1u) u = w0;
            if (dir_b) d = E.two_ws[BOTTOM] - w0;
            else if ((cd >> k) & 1u) d = w0;
            if (dir_l && x0 + k == 0) wl = E.two_ws[LEFT] - w0;
            else if ((cl >> k) & 1u) wl = w0;
            if (dir_r && x0 + k == nx - 1) wr = E.two_ws[RIGHT] - w0;
            else if ((cr >> k) & 1u) wr = w0;
            const T lap = ((u + d) + (wl + wr)) - (T)4 * w0;
            wdnew.v[k] = wdv.v[k] + a.g * lap;
            wn.v[k] = w0 + a.dt * wdnew.v[k];
        }
        T ac = (T)0;
        store_row(a, x0, j, wn, wdnew, ac);
        if (own) acc += ac;
        write_pads(a, x0, j, wn);
        dn = c;
        c = up;
        lc = lu;
        rc = ru;
        if (more) {
            sides(nxt, ln, rn);
            up = nxt;
            lu = ln;
            ru = rn;
            wdv = wdn;
        }
    }
    return acc;
}

// The grid is (column blocks of kThreads vectors) x (bands of kLineRows rows).
template <typename T>
__global__ void __launch_bounds__(kThreads) line_step_kernel(const StepArgs<T, T> a)
{
    constexpr int N = Vec<T>::N;
    constexpr int cols = kThreads * N;
    __shared__ CrackState sS;
    const int tid = threadIdx.x, lane = tid & 31;
    const int cb = blockIdx.x;
    const int x0 = (cb * kThreads + tid) * N;
    const int xw0 = (cb * kThreads + (tid & ~31)) * N;
    const int j0 = blockIdx.y * kLineRows, j1 = min(j0 + kLineRows, a.ny);
    const CrackParams &p = a.p;
    const CrackState *s_in = a.s_in;
    // the tip's cell, and the CTAs with sites within reach of the pending
    // crack step (a margin of one spacing beyond the two it needs)
    const int ti = (int)lo64((int64_t)p.nx - 1, s_in->r.tip_q >> kQBits);
    const int tj = (int)lo64((int64_t)p.ny - 1, s_in->r.tip_yq >> kQBits);
    const int c0 = cb * cols, c1 = c0 + cols - 1;
    const bool runner = c0 <= ti + 3 && c1 >= ti - 3 && j0 <= tj + 3 && j1 - 1 >= tj - 3;
    if (runner) {
        const bool commit = c0 <= ti && ti <= c1 && j0 <= tj && tj < j1;
        if (tid < 32) {
            if (tid == 0) sS = *s_in;
            __syncwarp();
            const bool pending = !sS.r.decided;   // not yet applied by a deferred crack step
            line_step_warp<T>(p, a.w_in, a.pitch, a.cut_h, a.cut_v, a.hist, sS, commit);
            if (tid == 0 && commit) {
                CrackState *o = a.s_out;
                const int64_t n = sS.step + 1;
                o->step = n;
                o->hist_n = sS.hist_n + (pending ? 1 : 0);
                o->i_first = sS.i_first;
                o->i_last = sS.i_last;
                o->r = sS.r;
                o->r.decided = 0;
                o->l = sS.l;
                for (int e = 0; e < 4; ++e)
                    o->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)p.dt) : 0.0;
            }
        }
        __syncthreads();   // this CTA's new cuts, for all of its threads
    }
    const EdgeValues<T> E = edge_values<T>(s_in);
    // warps wholly right of the lattice have nothing to load or store
    const T acc = xw0 < a.nx ? line_march<T>(a, E, x0, j0, j1) : (T)0;
    // a non-finite w (or wdot, which enters w) turns the sum of the first
    // element of each vector non-finite within a step or two
    if (__any_sync(0xffffffffu, !isfinite(acc)) && lane == 0) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
}

// The pending crack step before the host reads the state (one warp).
template <typename T>
__global__ void line_finalize_kernel(const FinalizeArgs<T> a)
{
    __shared__ CrackState sS;
    if (threadIdx.x == 0) sS = *a.st;
    __syncwarp();
    const bool pending = !sS.r.decided;
    line_step_warp<T>(a.p, a.w, a.pitch, a.cut_h, a.cut_v, a.hist, sS, true);
    if (threadIdx.x == 0) {
        if (pending && a.p.mode != CRACK_NONE) sS.hist_n += 1;
        *a.st = sS;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_line_step(const StepArgs<T, T> &a, cudaStream_t s)
{
    const dim3 grid((unsigned)a.ncb, (unsigned)((a.ny + kLineRows - 1) / kLineRows));
    line_step_kernel<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_line_finalize(const FinalizeArgs<T> &a, cudaStream_t s)
{
    line_finalize_kernel<T><<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_line_step<double>(const StepArgs<double, double> &, cudaStream_t);
template cudaError_t launch_line_step<float>(const StepArgs<float, float> &, cudaStream_t);
template cudaError_t launch_line_finalize<double>(const FinalizeArgs<double> &, cudaStream_t);
template cudaError_t launch_line_finalize<float>(const FinalizeArgs<float> &, cudaStream_t);

}  // namespace lbm
