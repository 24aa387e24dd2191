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
// link.  As in the step kernel, the crack step that follows step k - 1 is
// applied at the start of step k, here by one CTA of its own (block 0,
// scheduled first): it runs the crack step and then updates the sites within
// three spacings of the tip's cell -- the links an advance of less than one
// spacing severs have both ends within two spacings of the old tip.  The
// other CTAs march up the rows like the step kernel (16 bytes per site
// update) without reading cut words, skipping the 32-site groups that meet
// the band around the crack and the tip's box; after its march each CTA
// updates a share of those groups site by site with their severed links.
// No CTA waits for the crack step, and the cut bits the CTAs read are not
// changed during the launch.
#include "lbm_crack.cuh"
#include "lbm_internal.cuh"
#include "lbm_line.cuh"
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
                                   const uint32_t *cut_v, const TipState &E, int dir)
{
    const int lane = threadIdx.x & 31;
    const double r_min = p.r_min_fixed > 0.0 ? p.r_min_fixed : p.r0 / (1.0 - E.v_prev);   // eq. r(v)
    const double lo = r_min / p.dh, hi = (r_min + p.fit_width) / p.dh;
    const double tx = (double)E.tip_q * kTwoM32, ty = (double)E.tip_yq * kTwoM32;
    // the window lies behind the tip: along -c from the right end, along +c
    // from the left end of a two-tip crack
    const double sx = dir > 0 ? -p.dir_x : p.dir_x, sy = dir > 0 ? -p.dir_y : p.dir_y;
    const double ax = tx + lo * sx, bx = tx + hi * sx, ay = ty + lo * sy, by = ty + hi * sy;
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
            const double px = __dmul_rn((double)(dir > 0 ? E.tip_q - mx : mx - E.tip_q) * kTwoM32, p.dir_x);
            const double py = __dmul_rn((double)(dir > 0 ? E.tip_yq - my : my - E.tip_yq) * kTwoM32, p.dir_y);
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

// Steps (2)-(4) of the crack step for one end (dir = +1: the tip, growing
// along c; -1: the start of a two-tip crack, growing along -c), by one warp
// on the state S (shared memory), given that end's sums: K, the criterion,
// the advance (with the stop at the boundary), the severed links, the end's
// fields of S and, if `commit`, its history record at hist_n (x in tip /
// tipl, y in tipy / tipyl).
__device__ void line_apply_warp(const CrackParams &p, uint32_t *cut_h, uint32_t *cut_v, const History &hist,
                                CrackState &S, int dir, bool commit, const LineSums &c)
{
    const int lane = threadIdx.x & 31;
    TipState &E = dir > 0 ? S.r : S.l;
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
        const int64_t ax = __double2ll_rn(q * p.dir_x), ay = __double2ll_rn(q * p.dir_y);
        qx = dir > 0 ? px + ax : px - ax;
        qy = dir > 0 ? py + ay : py - ay;
        if (line_clamp(p, px, py, qx, qy)) { arrested = 1; flags |= FLAG_CLAMPED; }
    }
    const int grew = (qx != px || qy != py) ? 1 : 0;
    if (grew) {
        // sever every link the segment (px, py)-(qx, qy) meets: both ends of
        // such a link lie within one spacing of the segment
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
            if (dir > 0) {
                hist.K[h] = K;
                hist.v[h] = v;
                hist.tip[h] = qx;
                hist.tipy[h] = qy;
                hist.np[h] = c.np;
            } else {
                hist.Kl[h] = K;
                hist.vl[h] = v;
                hist.tipl[h] = qx;
                hist.tipyl[h] = qy;
                hist.npl[h] = c.np;
            }
        }
        E.decided = 1;
    }
    __syncwarp();
}

// The whole crack step by one warp, as Alg. 1 orders it: the criteria of
// both ends on the same state, then the right end's advance, then the left
// end's (the finalize kernel).
template <typename T>
__device__ void line_step_warp(const CrackParams &p, const T *w, int64_t P, uint32_t *cut_h, uint32_t *cut_v,
                               const History &hist, CrackState &S, bool commit)
{
    const int lane = threadIdx.x & 31;
    if (p.mode == CRACK_NONE || S.r.decided) {
        __syncwarp();
        if (lane == 0) { S.r.decided = 1; S.l.decided = 1; }
        __syncwarp();
        return;
    }
    const LineSums cr = line_eval_warp<T>(p, w, P, cut_h, cut_v, S.r, +1);
    LineSums cl{0.0, 0.0, 0.0, 0};
    if (p.two_tips) cl = line_eval_warp<T>(p, w, P, cut_h, cut_v, S.l, -1);
    line_apply_warp(p, cut_h, cut_v, hist, S, +1, commit, cr);
    if (p.two_tips) line_apply_warp(p, cut_h, cut_v, hist, S, -1, commit, cl);
}

// The pad images of the new value v of site (i, j) (free edges: the site's
// own value; periodic edges: the wrap-around value), as write_pads does for a
// row vector.
template <typename T, typename D>
__device__ __forceinline__ void site_pads(const StepArgs<T, D> &a, int i, int j, T v)
{
    const int nx = a.nx, ny = a.ny;
    const int64_t P = a.pitch;
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
        if (a.edge[BOTTOM] == EDGE_FREE) row[i - P] = v;
        else if (a.edge[BOTTOM] == EDGE_PERIODIC) a.w_out[(int64_t)ny * P + i] = v;
    }
    if (j == ny - 1) {
        if (a.edge[TOP] == EDGE_FREE) row[i + P] = v;
        else if (a.edge[TOP] == EDGE_PERIODIC) a.w_out[i - P] = v;
    }
}

// The update of one site with its severed links (the update of the march,
// site by site); returns whether the new w is finite.
template <typename T, typename D>
__device__ __forceinline__ bool site_update(const StepArgs<T, D> &a, const EdgeValues<T> &E, int i, int j)
{
    const int nx = a.nx, ny = a.ny, words = a.words;
    const int64_t P = a.pitch;
    const T *r0 = a.w_in + (int64_t)j * P;
    // every load first, so that they are in flight together
    const uint32_t *ch = a.cut_h + (int64_t)j * words, *cv = a.cut_v + (int64_t)j * words;
    const uint32_t hr_w = __ldcg(ch + (i >> 5));
    const uint32_t hl_w = i >= 1 ? __ldcg(ch + ((i - 1) >> 5)) : 0u;
    const uint32_t vu_w = j + 1 < ny ? __ldcg(cv + (i >> 5)) : 0u;
    const uint32_t vd_w = j >= 1 ? __ldcg(cv - words + (i >> 5)) : 0u;
    const T w0 = r0[i];
    T wl = r0[i - 1], wr = r0[i + 1], u = r0[i + P], d = r0[i - P];
    const int64_t o = (int64_t)j * P + i;
    T wdo;
    if constexpr (std::is_same<T, D>::value) wdo = a.wd[o];
    else wdo = WdIO<D>::get(a.wd + o, a.wd_inv);
    if (j == ny - 1 && a.edge[TOP] == EDGE_DIRICHLET) u = E.two_ws[TOP] - w0;
    else if ((vu_w >> (i & 31)) & 1u) u = w0;
    if (j == 0 && a.edge[BOTTOM] == EDGE_DIRICHLET) d = E.two_ws[BOTTOM] - w0;
    else if ((vd_w >> (i & 31)) & 1u) d = w0;
    if (i == 0 && a.edge[LEFT] == EDGE_DIRICHLET) wl = E.two_ws[LEFT] - w0;
    else if ((hl_w >> ((i - 1) & 31)) & 1u) wl = w0;
    if (i == nx - 1 && a.edge[RIGHT] == EDGE_DIRICHLET) wr = E.two_ws[RIGHT] - w0;
    else if ((hr_w >> (i & 31)) & 1u) wr = w0;
    const T lap = ((u + d) + (wl + wr)) - (T)4 * w0;
    const T wdn = wdo + a.g * lap;
    const T wn = w0 + a.dt * wdn;
    a.w_out[o] = wn;
    WdIO<D>::put(a.wd + o, wdn, a.wd_scale);
    site_pads(a, i, j, wn);
    return isfinite(wn);
}

// Which block updates a site.  The tip's box (the sites within three
// spacings of the tip's cell: every link the pending crack step can sever
// has both ends there) belongs to block 0.  Both ends of a severed link lie
// within one spacing of the crack (the polyline of the tips keeps to the
// line through the start along c within rounding) and at most one spacing
// behind the start or ahead of the tip.  Every group (kGroup consecutive
// sites of a row, aligned; a march thread's vector lies in one) that meets
// the band around that stretch of the line -- the points closer than 1.5
// spacings to the line, from 2 spacings behind the start to 2 ahead of the
// tip, widened by half a spacing along the row -- or the tip's box is
// claimed: the march leaves it, and claimed_groups updates it with its cuts.
// The groups of row j are those from sa(j) to sb(j), computed by one formula
// in explicitly rounded arithmetic, so that every block finds the same set.
constexpr int kGroup = 32;
struct Claims {
    int i0, i1, j0, j1;            // the tip's box
    int k0, k1, l0, l1;            // the left end's box (two-tip cracks; else empty)
    int r0, r1;                    // rows whose groups can be claimed
    float sx, sy, cx, cy;          // start, direction
    float t_lo, t_hi;              // the ends' distances along c from the start, minus / plus 2
    float inv_cx, inv_cy;          // 1 / c (0 where |c| is below 1e-6: the row is all in or all out)
};

__device__ __forceinline__ Claims claims(const CrackParams &p, const CrackState *s)
{
    Claims c;
    // the boxes of the sites within three spacings of each growing end's
    // cell (tips lie in [0, nx] x [0, ny])
    const int64_t ti = s->r.tip_q >> kQBits, tj = s->r.tip_yq >> kQBits;
    c.i0 = (int)hi64(0, ti - 3);
    c.i1 = (int)lo64(p.nx - 1, ti + 3);
    c.j0 = (int)hi64(0, tj - 3);
    c.j1 = (int)lo64(p.ny - 1, tj + 3);
    c.k0 = c.l0 = 1;
    c.k1 = c.l1 = 0;
    const int64_t lxq = p.two_tips ? s->l.tip_q : p.start_q, lyq = p.two_tips ? s->l.tip_yq : p.start_yq;
    if (p.two_tips) {
        const int64_t li = lxq >> kQBits, lj = lyq >> kQBits;
        c.k0 = (int)hi64(0, li - 3);
        c.k1 = (int)lo64(p.nx - 1, li + 3);
        c.l0 = (int)hi64(0, lj - 3);
        c.l1 = (int)lo64(p.ny - 1, lj + 3);
    }
    const int64_t ya = lo64(lyq, s->r.tip_yq) >> kQBits, yb = hi64(lyq, s->r.tip_yq) >> kQBits;
    c.r0 = (int)hi64(0, lo64(ya - 3, lo64(c.j0, p.two_tips ? c.l0 : c.j0)));
    c.r1 = (int)lo64(p.ny - 1, hi64(yb + 3, hi64(c.j1, p.two_tips ? c.l1 : c.j1)));
    c.sx = (float)((double)p.start_q * kTwoM32);
    c.sy = (float)((double)p.start_yq * kTwoM32);
    c.cx = (float)p.dir_x;
    c.cy = (float)p.dir_y;
    const float tx = (float)((double)s->r.tip_q * kTwoM32), ty = (float)((double)s->r.tip_yq * kTwoM32);
    c.t_hi = __fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(tx, c.sx), c.cx), __fmul_rn(__fsub_rn(ty, c.sy), c.cy)), 2.0f);
    const float ux = (float)((double)lxq * kTwoM32), uy = (float)((double)lyq * kTwoM32);
    c.t_lo = __fsub_rn(__fadd_rn(__fmul_rn(__fsub_rn(ux, c.sx), c.cx), __fmul_rn(__fsub_rn(uy, c.sy), c.cy)), 2.0f);
    c.inv_cx = fabsf(c.cx) < 1e-6f ? 0.0f : __frcp_rn(c.cx);
    c.inv_cy = fabsf(c.cy) < 1e-6f ? 0.0f : __frcp_rn(c.cy);
    return c;
}

__device__ __forceinline__ bool in_box(const Claims &c, int i, int j)
{
    return (i >= c.i0 && i <= c.i1 && j >= c.j0 && j <= c.j1) || (i >= c.k0 && i <= c.k1 && j >= c.l0 && j <= c.l1);
}

// Does group s (W sites wide) of row j meet one of the boxes?
__device__ __forceinline__ bool box_group(const Claims &c, int s, int j, int W)
{
    return (j >= c.j0 && j <= c.j1 && s >= c.i0 / W && s <= c.i1 / W) ||
           (j >= c.l0 && j <= c.l1 && c.k0 <= c.k1 && s >= c.k0 / W && s <= c.k1 / W);
}

// The groups of row j (W sites wide) that meet the band: sa .. sb (empty if
// sa > sb).
__device__ __forceinline__ void band_segs(const Claims &c, int j, int W, int nx, int &sa, int &sb)
{
    sa = 1;
    sb = 0;
    if (j < c.r0 || j > c.r1) return;
    const float y = __fsub_rn((float)j + 0.5f, c.sy);
    // |d| < 1.5 with d(x) = -(x - s_x) c_y + y c_x
    const float dy = __fmul_rn(y, c.cx);
    float xa = -3.0e38f, xb = 3.0e38f;
    if (c.inv_cy != 0.0f) {
        const float u = __fmul_rn(__fsub_rn(dy, 1.5f), c.inv_cy), v = __fmul_rn(__fadd_rn(dy, 1.5f), c.inv_cy);
        xa = __fadd_rn(c.sx, fminf(u, v));
        xb = __fadd_rn(c.sx, fmaxf(u, v));
    } else if (!(fabsf(dy) < 1.5f)) {
        return;
    }
    // t_lo < t < t_hi with t(x) = (x - s_x) c_x + y c_y
    const float ty = __fmul_rn(y, c.cy);
    if (c.inv_cx != 0.0f) {
        const float u = __fmul_rn(__fsub_rn(c.t_lo, ty), c.inv_cx), v = __fmul_rn(__fsub_rn(c.t_hi, ty), c.inv_cx);
        xa = fmaxf(xa, __fadd_rn(c.sx, fminf(u, v)));
        xb = fminf(xb, __fadd_rn(c.sx, fmaxf(u, v)));
    } else if (!(ty > c.t_lo && ty < c.t_hi)) {
        return;
    }
    // the columns whose centres lie within half a spacing of (xa, xb)
    const float fa = fmaxf(__fsub_rn(xa, 1.0f), 0.0f), fb = fminf(xb, (float)nx);
    if (!(fa <= fb)) return;
    const int ca = (int)fa, cb = min((int)fb, nx - 1);
    sa = ca / W;
    sb = cb / W;
}

__device__ __forceinline__ bool seg_claimed(const Claims &c, int s, int j, int W, int nx)
{
    if (box_group(c, s, j, W)) return true;
    int sa, sb;
    band_segs(c, j, W, nx, sa, sb);
    return s >= sa && s <= sb;
}

// Block 0: the pending crack step -- warp 0 the tip, warp 1 the left end of
// a two-tip crack; both criteria are evaluated before either end severs a
// link, as Alg. 1 orders them -- then the record and the next state (thread
// 0), then the ends' boxes with the cuts in force after it.
template <typename T, typename D>
__device__ void tip_cta(const StepArgs<T, D> &a, CrackState &sS, const EdgeValues<T> &E, const Claims &C)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    const CrackParams &p = a.p;
    if (tid == 0) sS = *a.s_in;
    __syncthreads();
    const bool pending = !sS.r.decided;   // not yet applied by a deferred crack step
    const bool active = p.mode != CRACK_NONE && pending;
    const int dir = warp == 0 ? +1 : -1;
    const bool mine = warp == 0 || (warp == 1 && p.two_tips);
    LineSums cs{0.0, 0.0, 0.0, 0};
    if (active && mine) cs = line_eval_warp<T>(p, a.w_in, a.pitch, a.cut_h, a.cut_v, dir > 0 ? sS.r : sS.l, dir);
    __syncthreads();   // both criteria on the state before either end severs a link
    if (active && mine) line_apply_warp(p, a.cut_h, a.cut_v, a.hist, sS, dir, true, cs);
    __syncthreads();
    if (tid < 32) {
        if (tid == 0) {
            CrackState *o = a.s_out;
            const int64_t n = sS.step + 1;
            o->step = n;
            o->hist_n = sS.hist_n + (pending ? 1 : 0);
            o->i_first = sS.i_first;
            o->i_last = sS.i_last;
            o->r = sS.r;
            o->r.decided = 0;
            o->l = sS.l;
            o->l.decided = 0;
            for (int e = 0; e < 4; ++e)
                o->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)p.dt) : 0.0;
        }
    }
    __syncthreads();   // the new cuts, for every thread of the CTA
    bool ok = true;
    const int ni = C.i1 - C.i0 + 1, nj = C.j1 - C.j0 + 1;
    for (int t = tid; t < ni * nj; t += blockDim.x) ok &= site_update(a, E, C.i0 + t % ni, C.j0 + t / ni);
    // the left end's box, less the sites of the tip's
    const int mi = C.k1 - C.k0 + 1, mj = C.l1 - C.l0 + 1;
    for (int t = tid; t < (mi > 0 ? mi * mj : 0); t += blockDim.x) {
        const int i = C.k0 + t % mi, j = C.l0 + t / mi;
        if (!(i >= C.i0 && i <= C.i1 && j >= C.j0 && j <= C.j1)) ok &= site_update(a, E, i, j);
    }
    if (!ok) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
}

// The claimed groups: every site outside the boxes of every claimed group.  The rows r0 .. r1, each cut into stretches of 16 groups, are taken
// in turn by the `nblk` march blocks after their march; a block finds the
// groups of its stretch that the band or a box claims (one evaluation of the
// band per stretch; its warps test four groups each) and updates them, a
// site per lane.  The cuts they read are not changed during the launch (new
// ones all lie in the boxes), and no march block writes a claimed site.
template <typename T, typename D>
__device__ void claimed_groups(const StepArgs<T, D> &a, const EdgeValues<T> &E, const Claims &C, int blk, int nblk)
{
    constexpr int kStretch = 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int ngroup = (a.nx + kGroup - 1) / kGroup, nstretch = (ngroup + kStretch - 1) / kStretch;
    const int items = (C.r1 - C.r0 + 1) * nstretch;
    bool ok = true;
    for (int q = blk; q < items; q += nblk) {
        const int j = C.r0 + q / nstretch, g0 = (q % nstretch) * kStretch, g1 = min(g0 + kStretch, ngroup) - 1;
        int sa, sb;
        band_segs(C, j, kGroup, a.nx, sa, sb);
        for (int t = warp; t <= g1 - g0; t += nwarp) {
            const int g = g0 + t;
            if (!((g >= sa && g <= sb) || box_group(C, g, j, kGroup))) continue;
            const int i = g * kGroup + lane;
            if (i < a.nx && !in_box(C, i, j)) ok &= site_update(a, E, i, j);
        }
    }
    if (!ok) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
}

// The march of a warp whose part of the band holds no edge row or column and
// no claimed site: the bare update.
template <typename T, typename D>
__device__ __forceinline__ T line_march_bare(const StepArgs<T, D> &a, int x0, int j0, int j1)
{
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t P = a.pitch;
    const T *win = a.w_in + x0;
    T *wout = a.w_out + x0;
    D *wdp = a.wd + x0;
    const T wd_inv = a.wd_inv, wd_scale = a.wd_scale;
    R dn, c, up, wdv;
    ldg_row(win + (int64_t)(j0 - 1) * P, dn);
    ldg_row(win + (int64_t)j0 * P, c);
    ldg_row(win + (int64_t)(j0 + 1) * P, up);
    WdIO<D>::load(wdp + (int64_t)j0 * P, wdv, wd_inv);
    T hl = (T)0, hr = (T)0;
    if (lane == 0) hl = win[(int64_t)j0 * P - 1];
    if (lane == 31) hr = win[(int64_t)j0 * P + N];
    const T g = a.g, dt = a.dt;
    T acc = (T)0;
    for (int j = j0; j < j1; ++j) {
        R nxt;
        typename WdIO<D>::Raw wdn;   // converted after this row's update, when it has arrived
        T hln = (T)0, hrn = (T)0;
        const bool more = j + 1 < j1;
        if (more) {
            ldg_row(win + (int64_t)(j + 2) * P, nxt);
            WdIO<D>::fetch(wdp + (int64_t)(j + 1) * P, wdn);
            if (lane == 0) hln = win[(int64_t)(j + 1) * P - 1];
            if (lane == 31) hrn = win[(int64_t)(j + 1) * P + N];
        }
        T lc = __shfl_up_sync(kFull, c.v[N - 1], 1), rc = __shfl_down_sync(kFull, c.v[0], 1);
        if (lane == 0) lc = hl;
        if (lane == 31) rc = hr;
        R wn, wdnew;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T wl = k == 0 ? lc : c.v[k - 1], wr = k == N - 1 ? rc : c.v[k + 1];
            const T lap = ((up.v[k] + dn.v[k]) + (wl + wr)) - (T)4 * c.v[k];
            wdnew.v[k] = wdv.v[k] + g * lap;
            wn.v[k] = c.v[k] + dt * wdnew.v[k];
        }
        stg_row(wout + (int64_t)j * P, wn);
        WdIO<D>::store(wdp + (int64_t)j * P, wdnew, wd_scale);
        acc += wn.v[0];
        dn = c;
        c = up;
        if (more) {
            up = nxt;
            WdIO<D>::unpack(wdn, wdv, wd_inv);
            hl = hln;
            hr = hrn;
        }
    }
    return acc;
}

// The march of the other warps: with EDGE, Dirichlet edges by
// anti-bounce-back and free and periodic edges through the pads (as the step
// kernel's edge warps); with CHECK, no store to a claimed group.  No cut
// word is read: every site next to a severed link lies in a claimed group.
template <typename T, typename D, bool EDGE, bool CHECK>
__device__ __forceinline__ T line_march_edge(const StepArgs<T, D> &a, const EdgeValues<T> &E, const Claims &C, int x0,
                                             int xw0, int j0, int j1)
{
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const int64_t P = a.pitch;
    const T *wb = a.w_in;
    const int grp = x0 / kGroup;
    R dn, c, up, wdv;
    ldg_row(wb + (int64_t)(j0 - 1) * P + x0, dn);
    ldg_row(wb + (int64_t)j0 * P + x0, c);
    ldg_row(wb + (int64_t)(j0 + 1) * P + x0, up);
    WdIO<D>::load(a.wd + x0 + (int64_t)j0 * P, wdv, a.wd_inv);
    T hl = (T)0, hr = (T)0;
    if (lane == 0) hl = wb[(int64_t)j0 * P + x0 - 1];
    if (lane == 31) hr = wb[(int64_t)j0 * P + x0 + N];
    T acc = (T)0;
    for (int j = j0; j < j1; ++j) {
        R nxt;
        typename WdIO<D>::Raw wdn;
        T hln = (T)0, hrn = (T)0;
        const bool more = j + 1 < j1;
        if (more) {
            ldg_row(wb + (int64_t)(j + 2) * P + x0, nxt);
            WdIO<D>::fetch(a.wd + x0 + (int64_t)(j + 1) * P, wdn);
            if (lane == 0) hln = wb[(int64_t)(j + 1) * P + x0 - 1];
            if (lane == 31) hrn = wb[(int64_t)(j + 1) * P + x0 + N];
        }
        T lc = __shfl_up_sync(kFull, c.v[N - 1], 1), rc = __shfl_down_sync(kFull, c.v[0], 1);
        if (lane == 0) lc = hl;
        if (lane == 31) rc = hr;
        if (!CHECK || !seg_claimed(C, grp, j, kGroup, nx)) {
            R wn, wdnew;
            if (EDGE) {
                row_update(a, E, x0, j, c, up, dn, wdv, lc, rc, 0u, 0u, wn, wdnew);
                if (x0 < nx) {
                    T ac = (T)0;
                    store_row(a, x0, j, wn, wdnew, ac);
                    acc += ac;
                    write_pads(a, x0, j, wn);
                }
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const T wl = k == 0 ? lc : c.v[k - 1], wr = k == N - 1 ? rc : c.v[k + 1];
                    const T lap = ((up.v[k] + dn.v[k]) + (wl + wr)) - (T)4 * c.v[k];
                    wdnew.v[k] = wdv.v[k] + a.g * lap;
                    wn.v[k] = c.v[k] + a.dt * wdnew.v[k];
                }
                stg_row(a.w_out + x0 + (int64_t)j * P, wn);
                WdIO<D>::store(a.wd + x0 + (int64_t)j * P, wdnew, a.wd_scale);
                acc += wn.v[0];
            }
        }
        dn = c;
        c = up;
        if (more) {
            up = nxt;
            WdIO<D>::unpack(wdn, wdv, a.wd_inv);
            hl = hln;
            hr = hrn;
        }
    }
    return acc;
}

// A 1-D grid: block 0 handles the tip (tip_cta), block 1 + cb + ncb * band
// marches column block cb of band `band` (p.band rows; bands as short as
// keeps every block resident at once) and then takes its share of the
// claimed groups.
template <typename T, typename D>
__device__ __forceinline__ void line_cta(const StepArgs<T, D> &a, int blk, CrackState &sS, Claims &sC,
                                         EdgeValues<T> &sE)
{
    constexpr int N = Vec<T>::N;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        sC = claims(a.p, a.s_in);
        sE = edge_values<T>(a.s_in);
    }
    __syncthreads();
    const EdgeValues<T> &E = sE;
    const Claims &C = sC;
    if (blk == 0) {
        tip_cta<T, D>(a, sS, E, C);
        return;
    }
    const int n_march = a.ncb * ((a.ny + a.p.band - 1) / a.p.band);
    const int u = blk - 1;
    const int cb = u % a.ncb, band = u / a.ncb;
    const int x0 = (cb * kThreads + tid) * N;
    const int xw0 = (cb * kThreads + (tid & ~31)) * N;
    const int j0 = band * a.p.band, j1 = min(j0 + a.p.band, a.ny);
    const int nx = a.nx, ny = a.ny;
    // warps wholly right of the lattice have nothing to load or store
    if (xw0 >= nx) {
        claimed_groups<T, D>(a, E, C, u, n_march);
        return;
    }
    // can the warp's part of the band hold an edge row or column, or a
    // claimed group: a box, or the band (the rectangle of the warp's sites
    // against the strip |d| < 1.5, t_lo < t < t_hi, with margins
    // beyond the half-spacing widening; d and t are linear, so their
    // extremes over the rectangle lie at its corners)?
    constexpr int W = 32 * N;
    const bool edge = xw0 == 0 || xw0 + W - 1 >= nx - 1 || j0 == 0 || j1 == ny;
    bool check = (j0 <= C.j1 && j1 - 1 >= C.j0 && xw0 + W - 1 >= (C.i0 / kGroup) * kGroup &&
                  xw0 <= (C.i1 / kGroup) * kGroup + kGroup - 1) ||
                 (C.k0 <= C.k1 && j0 <= C.l1 && j1 - 1 >= C.l0 && xw0 + W - 1 >= (C.k0 / kGroup) * kGroup &&
                  xw0 <= (C.k1 / kGroup) * kGroup + kGroup - 1);
    if (!check && j1 - 1 >= C.r0 && j0 <= C.r1) {
        const float xa = (float)xw0 + 0.5f - C.sx, xb = (float)(xw0 + W) - 0.5f - C.sx;
        const float ya = (float)j0 + 0.5f - C.sy, yb = (float)(j1 - 1) + 0.5f - C.sy;
        float dlo = 3.0e38f, dhi = -3.0e38f, tlo = 3.0e38f, thi = -3.0e38f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float x = (q & 1) ? xb : xa, y = (q & 2) ? yb : ya;
            const float d = -x * C.cy + y * C.cx, t = x * C.cx + y * C.cy;
            dlo = fminf(dlo, d);
            dhi = fmaxf(dhi, d);
            tlo = fminf(tlo, t);
            thi = fmaxf(thi, t);
        }
        check = !(dlo > 3.0f || dhi < -3.0f || thi < C.t_lo - 2.0f || tlo > C.t_hi + 2.0f);
    }
    T acc;
    if (edge) acc = check ? line_march_edge<T, D, true, true>(a, E, C, x0, xw0, j0, j1)
                          : line_march_edge<T, D, true, false>(a, E, C, x0, xw0, j0, j1);
    else acc = check ? line_march_edge<T, D, false, true>(a, E, C, x0, xw0, j0, j1) : line_march_bare<T, D>(a, x0, j0, j1);
    // a non-finite w (or wdot, which enters w) turns the sum of the first
    // element of each vector non-finite within a step or two
    if (__any_sync(0xffffffffu, !isfinite(acc)) && lane == 0) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
    claimed_groups<T, D>(a, E, C, u, n_march);
}

template <typename T, typename D>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2)
    line_step_kernel(const StepArgs<T, D> a)
{
    __shared__ CrackState sS;
    __shared__ Claims sC;                 // the claims and edge values, formed once per block
    __shared__ EdgeValues<T> sE;
    pdl_wait();
    pdl_trigger();
    line_cta<T, D>(a, blockIdx.x, sS, sC, sE);
}

// Many lattices with a crack in any direction in one launch: unit u is block
// u.cb of lattice u.inst's grid (0: the tip CTA, then its march blocks),
// run with the lattice's arguments for the current parity copied to shared
// memory first; the per-CTA code is the single-lattice kernel's, so each
// lattice ends bit-identical to its solo run.
template <typename T, typename D>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2)
    batch_line_kernel(const StepArgs<T, D> *descs, const BatchUnit *units, int par)
{
    __shared__ CrackState sS;
    __shared__ Claims sC;
    __shared__ EdgeValues<T> sE;
    __shared__ __align__(16) StepArgs<T, D> sa;
    pdl_wait();
    pdl_trigger();
    const BatchUnit u = units[blockIdx.x];
    const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + 2 * u.inst + par);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
    for (int q = threadIdx.x; q < (int)(sizeof(StepArgs<T, D>) / 4); q += kThreads) dst[q] = src[q];
    __syncthreads();
    line_cta<T, D>(sa, u.cb, sS, sC, sE);
}

// Is tabulated site (i, j) a boundary point now, i.e. is one of its links
// severed (read after the step, so the cuts of this step's crack step count)?
template <typename T, typename D>
__device__ __forceinline__ bool face_is_point(const StepArgs<T, D> &a, int i, int j)
{
    const int words = a.words;
    const uint32_t *ch = a.cut_h + (int64_t)j * words, *cv = a.cut_v + (int64_t)j * words;
    bool cut = (ch[i >> 5] >> (i & 31)) & 1u;
    if (i >= 1) cut |= (ch[(i - 1) >> 5] >> ((i - 1) & 31)) & 1u;
    if (j + 1 < a.ny) cut |= (cv[i >> 5] >> (i & 31)) & 1u;
    if (j >= 1) cut |= ((cv - words)[i >> 5] >> (i & 31)) & 1u;
    return cut;
}

// Report a point the rule does not support (a dropped stencil) or a solve
// that did not settle: FLAG_UNSUPPORTED in the state after this step, both
// ends (lbm_crack_state and lbm_crack_state_left read it).
template <typename T, typename D>
__device__ __forceinline__ void face_unsupported(const StepArgs<T, D> &a)
{
    atomicOr(&a.s_out->r.flags, (int32_t)FLAG_UNSUPPORTED);
    atomicOr(&a.s_out->l.flags, (int32_t)FLAG_UNSUPPORTED);
}

// The macroscopic rule on the faces of a crack in any direction (Sec. 3.1),
// after the march: chunk blockIdx.x of the table (see FaceChunk), one CTA
// each, a thread per item.  Each CTA gathers, for every item, in one
// parallel pass: whether it is a point, its current w (this step's update),
// the part of its sum over corners that are no table entry (fixed during the
// solve), its own site's weight and its coupled corners' weights and item
// indices -- all into shared memory.  A CTA whose own entries hold no point
// then leaves.  The others solve the points level by level from shared
// memory alone: w_B = base
// + sum over coupled corners of a_k w(corner) reads only lower levels (solved
// points, or the update of items that are no point) and its own site, whose
// weight (below 0.2) is solved by a scalar iteration from the update
// (monotone, so it settles).  Last, each CTA writes its own points' w_B,
// wdot_B = (w_B - w_B(t)) / dt and pad images.  Items that several chunks
// hold are computed alike in each.  The arithmetic is in the storage's type
// T (FP32 for FP32 storage: GB300's FP64 rate is a small fraction of its
// FP32 rate).
template <typename T, typename D>
__global__ void __launch_bounds__(kFaceItemsMax, 1) line_faces_chunk_kernel(const StepArgs<T, D> a, const FaceChunk *Cs,
                                                                         const FaceItem *I)
{
    extern __shared__ __align__(16) unsigned char face_smem[];
    __shared__ int slv[kFaceLevels + 1];
    pdl_wait();
    pdl_trigger();
    const int tid = threadIdx.x, nt = blockDim.x;
    const FaceChunk &C = Cs[blockIdx.x];
    const int64_t P = a.pitch;
    // the level offsets, read once (the level loop below must not wait on
    // a global load per level)
    for (int L = tid; L <= kFaceLevels; L += nt) slv[L] = C.lv[L];
    const int n = C.n;
    T *val = reinterpret_cast<T *>(face_smem);        // [n]
    T *base = val + n;                                 // [n]
    T *aself = base + n;                               // [n]
    T *ac = aself + n;                                 // [8 n] weights of the coupled corners
    int32_t *site = reinterpret_cast<int32_t *>(ac + 8 * n);  // [2 n] the item's (i, j)
    int16_t *kc = reinterpret_cast<int16_t *>(site + 2 * n);  // [8 n] coupled corners' items (-1: unused)
    uint8_t *act = reinterpret_cast<uint8_t *>(kc + 8 * n);   // [n] point (bit 0), own (bit 1), dropped (bit 2)
    int own_point = 0;
    for (int l = tid; l < n; l += nt) {
        // the whole record and w at all its corners first (unused corners name
        // the site itself), so the loads go out together rather than one
        // dependent chain per corner
        const FaceItem &it = I[C.off + l];
        const LineFace &f = it.rec;
        T wk[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) wk[k] = a.w_out[(int64_t)f.cj[k] * P + f.ci[k]];
        const bool point = face_is_point(a, f.i, f.j), own = it.f >= C.own_lo && it.f < C.own_hi;
        own_point |= point && own;
        act[l] = (point ? 1 : 0) | (own ? 2 : 0) | ((f.flags & FACE_DROPPED) ? 4 : 0);
        site[2 * l] = f.i;
        site[2 * l + 1] = f.j;
        val[l] = a.w_out[(int64_t)f.j * P + f.i];
        T b = (T)0, s = (T)0;
        int q = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const T ak = sizeof(T) == 4 ? (T)f.af[k] : (T)f.a[k];
            if (ak == (T)0) continue;
            const int m = it.kl[k];
            if (m == l) {
                s += ak;
            } else if (m >= 0) {
                ac[8 * l + q] = ak;
                kc[8 * l + q] = (int16_t)m;
                ++q;
            } else {
                b += ak * wk[k];
            }
        }
        for (int k = q; k < 8; ++k) kc[8 * l + k] = -1;
        base[l] = b;
        aself[l] = s;
    }
    // a CTA whose own entries hold no point has nothing to write
    if (!__syncthreads_or(own_point)) return;
    int stuck = 0;
    for (int L = 0; L < kFaceLevels; ++L) {
        const int lo = slv[L], hi = slv[L + 1];
        if (lo >= n) break;       // no item of this level or above
        if (lo == hi) continue;   // the same for every thread of the CTA
        for (int l = lo + tid; l < hi; l += nt) {
            if (!(act[l] & 1)) continue;
            T v = base[l];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int m = kc[8 * l + k];
                if (m < 0) break;
                v += ac[8 * l + k] * val[m];
            }
            const T s = aself[l];
            T x = val[l];
            int it_n = 0;
            for (; it_n < 64; ++it_n) {
                const T y = v + s * x;
                if (y == x) break;
                x = y;
            }
            stuck |= it_n == 64;
            val[l] = x;
        }
        __syncthreads();
    }
    const T inv_dt = (T)1 / a.dt;
    bool bad = false, drop = false;
    for (int l = tid; l < n; l += nt) {
        if ((act[l] & 3) != 3) continue;   // own points only
        const int i = site[2 * l], j = site[2 * l + 1];
        const int64_t o = (int64_t)j * P + i;
        const T wB = val[l];
        a.w_out[o] = wB;
        WdIO<D>::put(a.wd + o, (wB - a.w_in[o]) * inv_dt, a.wd_scale);
        site_pads(a, i, j, wB);
        bad |= !isfinite(wB);
        drop |= (act[l] & 4) != 0;
    }
    if (bad) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
    if (__syncthreads_or(drop || stuck) && tid == 0) face_unsupported(a);
}

// The macroscopic rule on the faces of a crack in any direction (Sec. 3.1),
// after the march, in one CTA (the form for tables the chunked solve does
// not take: a coupling deeper than kFaceLevels or a chunk too wide).  It lists the tabulated points whose site has
// a severed link (the list's order is immaterial: each sweep reads only the
// previous sweep's values) and, per point, sums once the terms of the
// corners that are not points (their w is this step's update, fixed during
// the solve) and notes the list positions of the corners that are.  Then it
// sweeps w_B = base + sum over the coupled corners of a_k w_B(corner), the
// values of two sweeps held in shared memory (in the scratch when the points
// outnumber it), until a sweep changes no bit (256 sweeps at most), and
// writes w_B and wdot_B = (w_B - w_B(t)) / dt.  Every corner but the point's
// own site lies farther from the line than the point (each is the point plus
// a lattice step in the normal's quadrant), so the coupling is acyclic apart
// from that one term; solving it within the sweep leaves as many sweeps as
// the coupling is deep.
constexpr int kFaceShared = 3008;   // points whose two sweep values fit in 48 KB of static shared memory

template <typename T, typename D>
__global__ void __launch_bounds__(1024) line_faces_kernel(const StepArgs<T, D> a, const LineFace *F, int nf,
                                                          FaceScratch z)
{
    __shared__ double sA[kFaceShared], sB[kFaceShared];
    __shared__ int n_act;
    pdl_wait();
    pdl_trigger();
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t P = a.pitch;
    if (tid == 0) n_act = 0;
    __syncthreads();
    for (int c = tid; c < nf; c += nt) {
        int q = -1;
        if (face_is_point(a, F[c].i, F[c].j)) {
            q = atomicAdd(&n_act, 1);
            z.list[q] = c;
        }
        z.pos[c] = q;
    }
    __syncthreads();
    const int na = n_act;
    double *cur = na <= kFaceShared ? sA : z.buf_a;
    double *nxt = na <= kFaceShared ? sB : z.buf_b;
    for (int q = tid; q < na; q += nt) {
        const LineFace &f = F[z.list[q]];
        double base = 0.0;
        uint32_t mask = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (f.a[k] == 0.0) continue;
            const int m = f.cand[k];
            const int pm = m >= 0 ? z.pos[m] : -1;
            if (pm >= 0) {
                mask |= 1u << k;
                z.kpos[8 * (int64_t)q + k] = pm;
            } else {
                base += f.a[k] * (double)a.w_out[(int64_t)f.cj[k] * P + f.ci[k]];
            }
        }
        z.base[q] = base;
        z.mask[q] = mask;
        cur[q] = (double)a.w_out[(int64_t)f.j * P + f.i];
    }
    __syncthreads();
    int changed = 1;
    for (int sweep = 0; sweep < 256 && changed; ++sweep) {
        changed = 0;
        for (int q = tid; q < na; q += nt) {
            const LineFace &f = F[z.list[q]];
            const uint32_t mask = z.mask[q];
            double v = z.base[q], a_self = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if ((mask >> k) & 1u) {
                    const int pk = z.kpos[8 * (int64_t)q + k];
                    if (pk == q) a_self += f.a[k];
                    else v += f.a[k] * cur[pk];
                }
            // the point's own site is a corner of its x_I cell (weight > 0,
            // below 1): solve x = v + a_self x for it here, by iteration from
            // its last value (monotone, so it settles in a few steps)
            double x = cur[q];
            for (int it = 0; it < 64; ++it) {
                const double y = v + a_self * x;
                if (y == x) break;
                x = y;
            }
            nxt[q] = x;
            changed |= x != cur[q];
        }
        // every read of cur and write of nxt of this sweep is done: the next
        // sweep reads nxt and overwrites cur
        changed = __syncthreads_or(changed);
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    const T inv_dt = (T)1 / a.dt;
    bool bad = false, drop = false;
    for (int q = tid; q < na; q += nt) {
        const int c = z.list[q];
        const int i = F[c].i, j = F[c].j;
        const int64_t o = (int64_t)j * P + i;
        const T wB = (T)cur[q];
        a.w_out[o] = wB;
        WdIO<D>::put(a.wd + o, (wB - a.w_in[o]) * inv_dt, a.wd_scale);
        site_pads(a, i, j, wB);
        bad |= !isfinite(wB);
        drop |= (F[c].flags & FACE_DROPPED) != 0;
    }
    if (bad) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
    // a dropped stencil in use, or 256 sweeps that still changed a value
    if ((drop || (changed && tid == 0))) face_unsupported(a);
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

template <typename T, typename D>
cudaError_t launch_line_faces(const StepArgs<T, D> &a, const LineFace *faces, int nf, double *scratch, cudaStream_t s)
{
    if (nf <= 0) return cudaSuccess;
    // the scratch holds kLineFaceScratch bytes per tabulated point
    FaceScratch z;
    z.buf_a = scratch;
    z.buf_b = z.buf_a + nf;
    z.base = z.buf_b + nf;
    z.list = reinterpret_cast<int32_t *>(z.base + nf);
    z.pos = z.list + nf;
    z.mask = reinterpret_cast<uint32_t *>(z.pos + nf);
    z.kpos = reinterpret_cast<int32_t *>(z.mask + nf);
    return launch_chained(line_faces_kernel<T, D>, dim3(1), dim3(1024), 0, s, a.chained != 0, a, faces, nf, z);
}

template <typename T, typename D>
cudaError_t launch_line_faces_chunked(const StepArgs<T, D> &a, const FaceChunk *chunks, int n_chunks,
                                      const FaceItem *items, cudaStream_t s)
{
    if (n_chunks <= 0) return cudaSuccess;
    // shared memory for kFaceItemsMax items: 11 T, 2 int32, 8 int16 and one byte each
    const size_t smem = (size_t)kFaceItemsMax * (11 * sizeof(T) + 2 * sizeof(int32_t) + 8 * sizeof(int16_t) + 1);
    cudaError_t e = cudaFuncSetAttribute(line_faces_chunk_kernel<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // a thread per item a CTA can hold: the gather's chains of dependent
    // loads (item record, face record, corner values) then go out in one round
    return launch_chained(line_faces_chunk_kernel<T, D>, dim3((unsigned)n_chunks), dim3(kFaceItemsMax), smem, s,
                          a.chained != 0, a, chunks, items);
}

template <typename T, typename D>
cudaError_t launch_line_step(const StepArgs<T, D> &a, cudaStream_t s)
{
    const unsigned bands = (unsigned)((a.ny + a.p.band - 1) / a.p.band);
    return launch_chained(line_step_kernel<T, D>, dim3(1u + (unsigned)a.ncb * bands), dim3(kThreads), 0, s,
                          a.chained != 0, a);
}

template <typename T, typename D>
cudaError_t launch_batch_line(const StepArgs<T, D> *descs, const BatchUnit *units, int n_units, int par, cudaStream_t s,
                              bool chained)
{
    if (n_units <= 0) return cudaSuccess;
    return launch_chained(batch_line_kernel<T, D>, dim3((unsigned)n_units), dim3(kThreads), 0, s, chained, descs, units,
                          par);
}

template <typename T>
cudaError_t launch_line_finalize(const FinalizeArgs<T> &a, cudaStream_t s)
{
    line_finalize_kernel<T><<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T, typename D>
const void *line_step_kernel_ptr()
{
    return reinterpret_cast<const void *>(&line_step_kernel<T, D>);
}

template const void *line_step_kernel_ptr<double, double>();
template const void *line_step_kernel_ptr<float, float>();
template const void *line_step_kernel_ptr<float, __nv_bfloat16>();
template const void *line_step_kernel_ptr<float, __half>();
template cudaError_t launch_line_faces<double, double>(const StepArgs<double, double> &, const LineFace *, int,
                                                      double *, cudaStream_t);
template cudaError_t launch_line_faces<float, float>(const StepArgs<float, float> &, const LineFace *, int, double *,
                                                    cudaStream_t);
template cudaError_t launch_line_faces<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> &, const LineFace *,
                                                            int, double *, cudaStream_t);
template cudaError_t launch_line_faces<float, __half>(const StepArgs<float, __half> &, const LineFace *, int, double *,
                                                     cudaStream_t);
template cudaError_t launch_line_faces_chunked<double, double>(const StepArgs<double, double> &, const FaceChunk *, int, const FaceItem *, cudaStream_t);
template cudaError_t launch_line_faces_chunked<float, float>(const StepArgs<float, float> &, const FaceChunk *, int, const FaceItem *, cudaStream_t);
template cudaError_t launch_line_faces_chunked<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> &, const FaceChunk *, int, const FaceItem *, cudaStream_t);
template cudaError_t launch_line_faces_chunked<float, __half>(const StepArgs<float, __half> &, const FaceChunk *, int, const FaceItem *, cudaStream_t);
template cudaError_t launch_line_step<double, double>(const StepArgs<double, double> &, cudaStream_t);
template cudaError_t launch_line_step<float, float>(const StepArgs<float, float> &, cudaStream_t);
template cudaError_t launch_line_step<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> &, cudaStream_t);
template cudaError_t launch_line_step<float, __half>(const StepArgs<float, __half> &, cudaStream_t);
template cudaError_t launch_batch_line<double, double>(const StepArgs<double, double> *, const BatchUnit *, int, int,
                                                  cudaStream_t, bool);
template cudaError_t launch_batch_line<float, float>(const StepArgs<float, float> *, const BatchUnit *, int, int,
                                                  cudaStream_t, bool);
template cudaError_t launch_batch_line<float, __nv_bfloat16>(const StepArgs<float, __nv_bfloat16> *, const BatchUnit *, int, int,
                                                  cudaStream_t, bool);
template cudaError_t launch_batch_line<float, __half>(const StepArgs<float, __half> *, const BatchUnit *, int, int,
                                                  cudaStream_t, bool);
template cudaError_t launch_line_finalize<double>(const FinalizeArgs<double> &, cudaStream_t);
template cudaError_t launch_line_finalize<float>(const FinalizeArgs<float> &, cudaStream_t);

}  // namespace lbm
