/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle for the lattice Boltzmann method
 * for antiplane shear with dynamic mode III crack propagation
 * (Schlueter-Kuhn et al., arXiv 2206.12412).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or helper with the CUDA library; the two are checked against
 * each other only through their outputs.
 *
 * What it implements, in the paper's order and notation:
 *   Sec. 3, eq. 2           D2Q5 velocity set c^0..c^4
 *   Sec. 3, eq. (LBE)       BGK collision f* = f - (dt/tau)(f - f_eq), then
 *                           streaming f(x + c dt, t + dt) = f*(x, t)
 *   Sec. 3, eq. (distrib-macro)  wdot = sum_a f^a
 *   Sec. 3, eq. (f-eq)      equilibrium, read as f_eq^k = g w (k = 1..4),
 *                           f_eq^0 = wdot - 4 g w, g = c_s^2 dt / dh^2, so that
 *                           sum_a f_eq^a = wdot and the scheme is the wave
 *                           equation with speed c_s (the printed scale is garbled)
 *   Sec. 3, eq. (integration)  w(t) = w(t - dt) + dt wdot(t)
 *   Sec. 3.1                links that a site misses: bounce-back on free
 *                           edges and crack faces, anti-bounce-back on
 *                           Dirichlet edges (link-local mode), or the
 *                           macroscopic rule of Sec. 3.1: a quadratic polynomial
 *                           through the boundary condition and w at two interior
 *                           points x_I, x_II (bilinear interpolation), evaluated
 *                           at x_B, then eq. (f-macro-bc) for the missing f^a
 *   Sec. 4.1, Alg. 1        CrackGrowth / CheckLinks (breadth-first search from
 *                           the neighbours of the previous boundary points) /
 *                           ProcessPoints
 *   Sec. 2.2, eq. (sif)     K = delta (mu/4) sqrt(2 pi / r) from the crack
 *                           opening of site pairs adjacent to the crack, at
 *                           r in [r_min, r_min + w_fit) (Sec. 4.2), least
 *                           squares over the pairs when w_fit > dh
 *   Sec. 4.2, eq. (r(v))    r_min = r0 / (1 - v)
 *   Sec. 4.2, eq. (v-tanh)  v = v_max tanh(sqrt((K/K_C)^4 - 1)), K > K_C
 *
 * Readings where the paper is silent or garbled (each one also listed in the
 * design notes of the repository):
 *   - sites sit at cell centres ((i + 1/2) dh, (j + 1/2) dh); outer edges and
 *     the crack line y = jc dh lie on half links;
 *   - the initial state is w = wdot = 0 unless set; f is set to f_eq(w, wdot);
 *   - a Dirichlet edge value w*(t_n) enters the step t_n -> t_n+1;
 *   - "intersects" is closed-segment intersection, tested exactly on a fixed
 *     point grid of 2^-32 dh; the tip is kept on that grid and every advance
 *     is rounded to nearest (ties to even) onto it;
 *   - r is measured along the crack from the tip, phi = +-pi, the window is
 *     half open; delta = w(above) - w(below), the criterion uses |K|;
 *   - r_min uses the v of the previous step (0 while arrested);
 *   - the tip stops (and stays) at the far edge x = nx dh, where the crack
 *     has severed every link of its row and split the body;
 *   - with the macroscopic rule on the outer edges too (Sec. 5.2), an edge
 *     site's polynomial lies along the edge's inward normal (x_I, x_II are
 *     the next two sites); a corner between two such edges follows its
 *     Dirichlet edge, or the bottom / top edge when both are of one kind;
 *     a site next to a severed crack link follows the crack face; the
 *     Dirichlet value is w*(t_n+1), the time of the unknown w_B; the system
 *     S w_B = R couples the boundary points only through interior points
 *     that are boundary points themselves and is solved exactly by sweeps
 *     until a sweep changes no bit;
 *   - a straight crack in any direction (Sec. 4.1) runs from its start
 *     through its initial tip and grows along that direction c: each
 *     component of Delta a c is rounded to the grid, so the crack is the
 *     polyline of the tips, every segment tested exactly; its pairs for K
 *     are the ends of the severed links, at r = (x_tip - m) . c from the
 *     link midpoint m, with delta = w(left of c) - w(right of c); the tip
 *     stops where it meets the body's boundary; the faces are link-local;
 *     with two growing ends the start is the left end, growing along -c,
 *     with r = (m - x_tip) . c and the same delta; with the macroscopic
 *     rule on its faces a boundary point takes the normal of the line (its
 *     x_I, x_II never reach across the crack), and the sweeps of the
 *     boundary solve run until no bit changes (256 at most).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 32 /* fixed point: 1 dh = 2^32 units */
#define ORC_PI 3.14159265358979323846

/* ORC_HALO: a bottom or top edge inside a lattice split into row slabs; each
 * distribution that crosses it into the slab (D2Q5: the one along y; D2Q9:
 * that one and the two diagonals) is the neighbouring slab's post-collision
 * value at the link's source site, handed over between the collision and the
 * streaming (orc_collide / orc_fs_row / orc_set_halo / orc_finish_step). */
enum { ORC_FREE = 0, ORC_DIRICHLET = 1, ORC_PERIODIC = 2, ORC_HALO = 3 };
enum { ORC_LEFT = 0, ORC_RIGHT = 1, ORC_BOTTOM = 2, ORC_TOP = 3 };
enum { ORC_BC_BOUNCEBACK = 0, ORC_BC_MACROSCOPIC = 1 };
enum { ORC_CRACK_NONE = 0, ORC_CRACK_STATIONARY = 1, ORC_CRACK_PRESCRIBED = 2, ORC_CRACK_KCRIT = 3 };
enum { ORC_LOAD_ZERO = 0, ORC_LOAD_LINEAR = 1, ORC_LOAD_SIN2 = 2, ORC_LOAD_HALFSINE = 3,
       ORC_LOAD_SERIES = 4, ORC_LOAD_CONST = 5 };
enum { ORC_FLAG_CLAMPED = 1, ORC_FLAG_UNSUPPORTED = 2, ORC_FLAG_NONFINITE = 4 };

typedef struct {
    int32_t nx, ny;
    double dh, dt;
    int32_t edge[4];     /* left, right, bottom, top */
    double rho, mu;
    double omega;        /* dt / tau; the paper fixes tau = dt */
    int32_t bc_mode;
    int32_t crack_mode;
    int32_t jc;          /* the crack lies on y = jc * dh */
    double x_start, x_tip;
    double v_rel, K_C, v_max, r0, r_min_fixed, fit_width;
    int32_t load_kind[4];
    double load_amp[4], load_t[4];
    const double *load_series[4];
    int64_t load_n[4];
    int64_t hist_cap;
    int32_t two_tips;    /* both ends of the crack grow (the left one towards -x) */
    int32_t edge_macro;  /* the macroscopic rule (Sec. 3.1) on the outer edges too */
    int32_t q;           /* velocity set: 5 (D2Q5, Sec. 3) or 9 (D2Q9) */
    int32_t pad_;
    int32_t line;        /* a straight crack in any direction, from (x_start, y_start) through (x_tip, y_tip) */
    int32_t pad2_;
    double y_start, y_tip;
} orc_config;

typedef struct {
    int32_t site;
    int32_t nI, idxI[4];
    double wI[4];
    int32_t nII, idxII[4];
    double wII[4];
    double sB, sI, sII;  /* distances from the crack face along the normal */
} orc_bpoint;

/* A boundary point of an outer edge under the macroscopic rule: its site,
 * the two sites x_I, x_II one and two spacings inside along the inward
 * normal of edge `edge`, and the rule (0: traction free, 1: Dirichlet). */
typedef struct {
    int32_t site, I, II, rule, edge;
} orc_epoint;

typedef struct {
    orc_config c;
    int64_t step;
    double cs, g;
    int Q;               /* 5 or 9 distributions */
    double *f[9], *fs[9], *w, *w_old;
    uint8_t *cut_h;      /* link (i,j)-(i+1,j), i = nx-1 is the periodic wrap */
    uint8_t *cut_v;      /* link (i,j)-(i,j+1), j = ny-1 is the periodic wrap */
    uint8_t *cut_d1;     /* D2Q9: link (i,j)-(i+1,j+1) */
    uint8_t *cut_d2;     /* D2Q9: link (i+1,j)-(i,j+1) */
    int64_t start_q, tip_q, clamp_q;
    int64_t start_yq, tip_yq;   /* y of the crack's start and tip (y = jc dh for the crack along +x) */
    double dir_x, dir_y;        /* unit direction of growth */
    int64_t *htipy, *htipyl;
    double v_prev, K_last;
    int32_t npairs_last, flags, arrested_for_good;
    int32_t *bprev, nbprev;
    /* the left tip (two_tips): position, speed memory, last K, arrest, B_prev */
    int64_t ltip_q, ltip_yq;
    double lv_prev, lK_last;
    int32_t lnpairs_last, larrested;
    int32_t *lbprev, nlbprev;
    double *hKl, *hvl;
    int64_t *htipl;
    int32_t *hnpl, *hgrowl;
    orc_epoint *ep;      /* outer-edge boundary points (edge_macro) */
    int32_t nep;
    orc_bpoint *bl;
    int32_t nbl, capbl;
    uint8_t *is_bpoint;
    int64_t hist_n;
    double *hK, *hv;
    int64_t *htip;
    int32_t *hnp, *hgrow;
    int32_t *queue;
    uint8_t *inq, *visited;
    double *series[4];
    int32_t threads;     /* OpenMP threads of the per-site loops (1 unless set) */
    double *halo[2][3];  /* ORC_HALO edges: the neighbour's boundary row of f*^a for each direction a
                            arriving at row 0 (2, then 5, 6) / at row ny-1 (4, then 7, 8), nx each */
} orc_state;

/* Lattice velocities in units of c = dh/dt: D2Q5 (Sec. 3, eq. 2) uses
 * 0..4; D2Q9 adds the diagonals 5..8. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Equilibrium weight of a moving direction, in units of g.  D2Q5: 1.  D2Q9:
 * 2/3 along the axes and 1/6 along the diagonals, the weights of the
 * isotropic nine-point Laplacian; the diagonal neighbours lie sqrt(2) dh away,
 * so the axis weight plus twice the diagonal weight is 1 and the wave speed
 * stays c_s. */
static double weight(const orc_state *s, int a)
{
    if (s->Q == 5) return 1.0;
    return a <= 4 ? 2.0 / 3.0 : 1.0 / 6.0;
}

static int64_t qone(void) { return (int64_t)1 << ORC_Q; }

/* ------------------------------------------------------------------ loading */

/* Boundary value w*(t) of a Dirichlet edge.
 * LINEAR: ramp amp * min(t / t_ramp, 1).
 * SIN2:   amp * sin^2(pi t / (2 t0)) for t < t0, then amp (Sec. 5.1).
 * HALFSINE: amp * sin(pi t / T) for t < T, then 0 (Sec. 5.2).
 * SERIES: series[n] at step n, last value afterwards. */
static double load_value(const orc_state *s, int e, int64_t n)
{
    const orc_config *c = &s->c;
    double t = (double)n * c->dt;
    double a = c->load_amp[e], T = c->load_t[e];
    switch (c->load_kind[e]) {
    case ORC_LOAD_LINEAR:
        if (T <= 0.0 || t >= T) return a;
        return a * (t / T);
    case ORC_LOAD_SIN2: {
        if (T <= 0.0 || t >= T) return a;
        double sn = sin(ORC_PI * t / (2.0 * T));
        return a * sn * sn;
    }
    case ORC_LOAD_HALFSINE:
        if (t >= T) return 0.0;
        return a * sin(ORC_PI * t / T);
    case ORC_LOAD_SERIES:
        if (c->load_n[e] <= 0) return 0.0;
        return s->series[e][n < c->load_n[e] ? n : c->load_n[e] - 1];
    case ORC_LOAD_CONST:
        return a;
    default:
        return 0.0;
    }
}

/* -------------------------------------------------------------- equilibrium */

/* Equilibrium distributions for the wave equation (Sec. 3, eq. f-eq), in the
 * reading f_eq^k = g w for the four moving directions and
 * f_eq^0 = wdot - 4 g w for the rest direction, g = c_s^2 dt / dh^2. */
static void equilibrium(double w, double wdot, double g, double feq[5])
{
    feq[0] = wdot - 4.0 * g * w;
    for (int a = 1; a < 5; ++a) feq[a] = g * w;
}

void orc_equilibrium(double w, double wdot, double g, double *feq5) { equilibrium(w, wdot, g, feq5); }

/* The same for the lattice of s: f_eq^a = weight_a g w (a >= 1), f_eq^0 =
 * wdot minus their sum, so that sum_a f_eq^a = wdot. */
static void equilibrium_q(const orc_state *s, double w, double wdot, double feq[9])
{
    double rest = wdot;
    for (int a = 1; a < s->Q; ++a) {
        feq[a] = weight(s, a) * s->g * w;
        rest -= feq[a];
    }
    feq[0] = rest;
}

/* ------------------------------------------------------------------ geometry */

static int64_t site_cx_q(int i) { return (int64_t)(2 * i + 1) << (ORC_Q - 1); }

static int orient(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy)
{
    __int128 v = (__int128)(bx - ax) * (__int128)(cy - ay) - (__int128)(by - ay) * (__int128)(cx - ax);
    return (v > 0) - (v < 0);
}

static int in_box(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py)
{
    int64_t lox = ax < bx ? ax : bx, hix = ax < bx ? bx : ax;
    int64_t loy = ay < by ? ay : by, hiy = ay < by ? by : ay;
    return px >= lox && px <= hix && py >= loy && py <= hiy;
}

/* Closed-segment intersection of p1p2 and q1q2, exact (orientation tests). */
int orc_segments_intersect(int64_t p1x, int64_t p1y, int64_t p2x, int64_t p2y,
                           int64_t q1x, int64_t q1y, int64_t q2x, int64_t q2y)
{
    int d1 = orient(q1x, q1y, q2x, q2y, p1x, p1y);
    int d2 = orient(q1x, q1y, q2x, q2y, p2x, p2y);
    int d3 = orient(p1x, p1y, p2x, p2y, q1x, q1y);
    int d4 = orient(p1x, p1y, p2x, p2y, q2x, q2y);
    if (d1 * d2 < 0 && d3 * d4 < 0) return 1;
    if (d1 == 0 && in_box(q1x, q1y, q2x, q2y, p1x, p1y)) return 1;
    if (d2 == 0 && in_box(q1x, q1y, q2x, q2y, p2x, p2y)) return 1;
    if (d3 == 0 && in_box(p1x, p1y, p2x, p2y, q1x, q1y)) return 1;
    if (d4 == 0 && in_box(p1x, p1y, p2x, p2y, q2x, q2y)) return 1;
    return 0;
}

/* Link between site k and its neighbour in direction a (a = 1..Q-1).
 * Returns the neighbour index, or -1 if the link leaves a non-periodic
 * domain.  *cut points at the severed flag of the link; *wrap is set when the
 * link crosses a periodic edge (such a link lies outside the body's interior
 * and no crack inside the body intersects it). */
static int32_t link_of_w(const orc_state *s, int32_t k, int a, uint8_t **cut, int *wrap)
{
    int nx = s->c.nx, ny = s->c.ny;
    int i = k % nx, j = k / nx;
    int ni = i + CX[a], nj = j + CY[a];
    *wrap = 0;
    if (ni < 0 || ni >= nx) {
        int e = ni < 0 ? ORC_LEFT : ORC_RIGHT;
        if (s->c.edge[e] != ORC_PERIODIC) return -1;
        ni = (ni + nx) % nx;
        *wrap = 1;
    }
    if (nj < 0 || nj >= ny) {
        int e = nj < 0 ? ORC_BOTTOM : ORC_TOP;
        if (s->c.edge[e] != ORC_PERIODIC) return -1;
        nj = (nj + ny) % ny;
        *wrap = 1;
    }
    /* the flag of an axis link is stored at the site from which it points in
     * +x / +y, that of a diagonal link at the lower-left corner of its cell */
    if (a == 1) *cut = &s->cut_h[j * nx + i];
    else if (a == 3) *cut = &s->cut_h[nj * nx + ni];
    else if (a == 2) *cut = &s->cut_v[j * nx + i];
    else if (a == 4) *cut = &s->cut_v[nj * nx + ni];
    else if (a == 5) *cut = &s->cut_d1[j * nx + i];
    else if (a == 7) *cut = &s->cut_d1[nj * nx + ni];
    else if (a == 6) *cut = &s->cut_d2[j * nx + ni];
    else *cut = &s->cut_d2[nj * nx + i];
    return nj * nx + ni;
}

static int32_t link_of(const orc_state *s, int32_t k, int a, uint8_t **cut)
{
    int wrap;
    return link_of_w(s, k, a, cut, &wrap);
}

/* The outer edge whose rule applies to the missing link of site k in
 * direction b: the edge it crosses; a diagonal link through a corner of the
 * body follows the Dirichlet edge if just one of the two is Dirichlet, else
 * the bottom / top edge. */
static int missing_edge(const orc_state *s, int32_t k, int b)
{
    int nx = s->c.nx, ny = s->c.ny;
    int ni = k % nx + CX[b], nj = k / nx + CY[b];
    int ex = (ni < 0 || ni >= nx) && s->c.edge[ni < 0 ? ORC_LEFT : ORC_RIGHT] != ORC_PERIODIC
                 ? (ni < 0 ? ORC_LEFT : ORC_RIGHT) : -1;
    int ey = (nj < 0 || nj >= ny) && s->c.edge[nj < 0 ? ORC_BOTTOM : ORC_TOP] != ORC_PERIODIC
                 ? (nj < 0 ? ORC_BOTTOM : ORC_TOP) : -1;
    if (ex >= 0 && ey >= 0) {
        /* across a row slab's boundary the lattice goes on: the link leaves
         * the body through the left / right edge alone */
        if (s->c.edge[ey] == ORC_HALO) return ex;
        return (s->c.edge[ex] == ORC_DIRICHLET && s->c.edge[ey] != ORC_DIRICHLET) ? ex : ey;
    }
    return ex >= 0 ? ex : ey;
}

/* Row slabs: the directions that cross a slab's boundary, in the order the
 * boundary rows are handed over: upwards (across a top edge, arriving at the
 * next slab's row 0) 2, 5, 6; downwards 4, 7, 8 (D2Q5: 2 / 4 alone). */
static const int HALO_UP[3] = {2, 5, 6}, HALO_DOWN[3] = {4, 7, 8};
static int halo_slot(int a) { return (a == 2 || a == 4) ? 0 : (a == 5 || a == 7) ? 1 : 2; }

/* ------------------------------------------------------------ state set-up */

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

void orc_destroy(orc_state *s)
{
    if (!s) return;
    for (int a = 0; a < 9; ++a) { free(s->f[a]); free(s->fs[a]); }
    free(s->w); free(s->w_old); free(s->cut_h); free(s->cut_v); free(s->cut_d1); free(s->cut_d2);
    free(s->bprev); free(s->bl); free(s->is_bpoint);
    free(s->hK); free(s->hv); free(s->htip); free(s->hnp); free(s->hgrow);
    free(s->ep);
    free(s->lbprev); free(s->hKl); free(s->hvl); free(s->htipl); free(s->htipy); free(s->htipyl); free(s->hnpl); free(s->hgrowl);
    free(s->queue); free(s->inq); free(s->visited);
    for (int e = 0; e < 4; ++e) free(s->series[e]);
    for (int e = 0; e < 2; ++e)
        for (int d = 0; d < 3; ++d) free(s->halo[e][d]);
    free(s);
}

static void add_bpoint(orc_state *s, int32_t k);
static int build_edge_points(orc_state *s);

/* Cut every link the initial crack segment intersects (brute force over all
 * links) and register both end points as boundary points; they form B_prev
 * for the first CheckLinks. */
static void initial_crack(orc_state *s)
{
    int nx = s->c.nx, ny = s->c.ny;
    int32_t *B = malloc(sizeof(int32_t) * 4 * (size_t)nx * ny);
    int nB = 0;
    static const int ONCE[4] = {1, 2, 5, 6};   /* each link once: +x, +y and the two upward diagonals */
    for (int32_t k = 0; k < nx * ny; ++k) {
        for (int q = 0; q < (s->Q == 9 ? 4 : 2); ++q) {
            int a = ONCE[q], wrap;
            uint8_t *cut;
            int32_t m = link_of_w(s, k, a, &cut, &wrap);
            if (m < 0 || wrap) continue;
            int i = k % nx, j = k / nx, mi = m % nx, mj = m / nx;
            if (orc_segments_intersect(site_cx_q(i), site_cx_q(j), site_cx_q(mi), site_cx_q(mj),
                                       s->start_q, s->start_yq, s->tip_q, s->tip_yq)) {
                *cut = 1;
                B[nB++] = k;
                B[nB++] = m;
            }
        }
    }
    s->nbprev = 0;
    for (int b = 0; b < nB; ++b) {
        int dup = 0;
        for (int q = 0; q < s->nbprev; ++q) dup |= s->bprev[q] == B[b];
        if (!dup) s->bprev[s->nbprev++] = B[b];
    }
    if (!s->c.line || s->c.bc_mode == ORC_BC_MACROSCOPIC)
        for (int b = 0; b < s->nbprev; ++b) add_bpoint(s, s->bprev[b]);
    free(B);
}

/* A crack in any direction (Sec. 4.1: the crack is a line independent of
 * the lattice, growing along a given direction): the start and the tip on
 * the fixed-point grid, the unit direction from the one to the other, and
 * the checks that the segment lies in the body [0, nx dh] x [0, ny dh] and
 * that its line passes through no site centre (a site on the crack would
 * be neither above nor below it).  The direction's components are formed
 * without fused multiply-adds (volatile products), so that every
 * implementation of this reading rounds them alike. */
static int line_setup(orc_state *s)
{
    const orc_config *c = &s->c;
    s->start_q = llrint(c->x_start / c->dh * (double)qone());
    s->start_yq = llrint(c->y_start / c->dh * (double)qone());
    s->tip_q = llrint(c->x_tip / c->dh * (double)qone());
    s->tip_yq = llrint(c->y_tip / c->dh * (double)qone());
    int64_t X = (int64_t)c->nx << ORC_Q, Y = (int64_t)c->ny << ORC_Q;
    if (s->start_q < 0 || s->start_q > X || s->tip_q < 0 || s->tip_q > X) return 0;
    if (s->start_yq < 0 || s->start_yq > Y || s->tip_yq < 0 || s->tip_yq > Y) return 0;
    if (s->start_q == s->tip_q && s->start_yq == s->tip_yq) return 0;
    volatile double dx = (double)(s->tip_q - s->start_q), dy = (double)(s->tip_yq - s->start_yq);
    volatile double xx = dx * dx, yy = dy * dy;
    double len = sqrt(xx + yy);
    s->dir_x = dx / len;
    s->dir_y = dy / len;
    for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i)
            if (orient(s->start_q, s->start_yq, s->tip_q, s->tip_yq, site_cx_q(i), site_cx_q(j)) == 0) return 0;
    return 1;
}

orc_state *orc_create(const orc_config *cfg)
{
    if (cfg->nx < 1 || cfg->ny < 1 || !(cfg->dh > 0) || !(cfg->dt > 0)) return NULL;
    int Q = cfg->q == 0 ? 5 : cfg->q;
    if (Q != 5 && Q != 9) return NULL;
    /* a crack in any direction is built for D2Q5 (link-local faces, or the
     * macroscopic rule on the crack faces only); its K window must lie more
     * than half a spacing behind the tip (the links a step severs have their
     * midpoints at most that far behind the old tip) */
    if (cfg->line) {
        if (Q != 5 || cfg->edge_macro || cfg->crack_mode == ORC_CRACK_NONE)
            return NULL;
        double rmin = cfg->r_min_fixed > 0.0 ? cfg->r_min_fixed : cfg->r0;
        if (!(rmin > 0.5 * cfg->dh)) return NULL;
    }
    /* halo edges (row slabs): bottom / top only, not with the macroscopic
     * rule on the outer edges, nor a crack in any direction */
    for (int e = 0; e < 4; ++e) {
        if (cfg->edge[e] != ORC_HALO) continue;
        if ((e != ORC_BOTTOM && e != ORC_TOP) || cfg->edge_macro || cfg->line) return NULL;
    }
    orc_state *s = xcalloc(1, sizeof(orc_state));
    s->c = *cfg;
    s->Q = Q;
    size_t n = (size_t)cfg->nx * cfg->ny;
    for (int e = 0; e < 2; ++e)
        for (int d = 0; d < 3; ++d) s->halo[e][d] = xcalloc((size_t)cfg->nx, sizeof(double));
    s->cs = sqrt(cfg->mu / cfg->rho);
    s->g = s->cs * s->cs * cfg->dt / (cfg->dh * cfg->dh);
    for (int a = 0; a < Q; ++a) { s->f[a] = xcalloc(n, sizeof(double)); s->fs[a] = xcalloc(n, sizeof(double)); }
    s->w = xcalloc(n, sizeof(double));
    s->w_old = xcalloc(n, sizeof(double));
    s->cut_h = xcalloc(n, 1);
    s->cut_v = xcalloc(n, 1);
    s->cut_d1 = xcalloc(n, 1);
    s->cut_d2 = xcalloc(n, 1);
    s->is_bpoint = xcalloc(n, 1);
    s->bprev = xcalloc(n, sizeof(int32_t));
    s->lbprev = xcalloc(n, sizeof(int32_t));
    s->capbl = 64;
    s->bl = xcalloc((size_t)s->capbl, sizeof(orc_bpoint));
    s->queue = xcalloc(8 * n + 8, sizeof(int32_t));
    s->inq = xcalloc(n, 1);
    s->visited = xcalloc(n, 1);
    s->hist_n = 0;
    int64_t hc = cfg->hist_cap > 0 ? cfg->hist_cap : 1;
    s->hK = xcalloc((size_t)hc, sizeof(double));
    s->hv = xcalloc((size_t)hc, sizeof(double));
    s->htip = xcalloc((size_t)hc, sizeof(int64_t));
    s->hnp = xcalloc((size_t)hc, sizeof(int32_t));
    s->hgrow = xcalloc((size_t)hc, sizeof(int32_t));
    s->hKl = xcalloc((size_t)hc, sizeof(double));
    s->hvl = xcalloc((size_t)hc, sizeof(double));
    s->htipl = xcalloc((size_t)hc, sizeof(int64_t));
    s->htipy = xcalloc((size_t)hc, sizeof(int64_t));
    s->htipyl = xcalloc((size_t)hc, sizeof(int64_t));
    s->hnpl = xcalloc((size_t)hc, sizeof(int32_t));
    s->hgrowl = xcalloc((size_t)hc, sizeof(int32_t));
    for (int e = 0; e < 4; ++e) {
        if (cfg->load_kind[e] == ORC_LOAD_SERIES && cfg->load_n[e] > 0) {
            s->series[e] = malloc(sizeof(double) * (size_t)cfg->load_n[e]);
            memcpy(s->series[e], cfg->load_series[e], sizeof(double) * (size_t)cfg->load_n[e]);
        }
        s->c.load_series[e] = NULL;
    }
    /* the initial state: w = wdot = 0, f = f_eq(0, 0) = 0 */
    s->v_prev = cfg->crack_mode == ORC_CRACK_PRESCRIBED ? cfg->v_rel : 0.0;
    s->clamp_q = (int64_t)cfg->nx << ORC_Q;
    if (cfg->crack_mode != ORC_CRACK_NONE) {
        s->start_q = llrint(cfg->x_start / cfg->dh * (double)qone());
        s->tip_q = llrint(cfg->x_tip / cfg->dh * (double)qone());
        s->start_yq = s->tip_yq = (int64_t)cfg->jc << ORC_Q;
        s->dir_x = 1.0;
        s->dir_y = 0.0;
        if (cfg->line && !line_setup(s)) {
            orc_destroy(s);
            return NULL;
        }
        s->ltip_q = s->start_q;
        s->ltip_yq = s->start_yq;
        s->lv_prev = s->v_prev;
        initial_crack(s);
        /* both tips start their CheckLinks from the initial boundary points */
        memcpy(s->lbprev, s->bprev, sizeof(int32_t) * (size_t)s->nbprev);
        s->nlbprev = s->nbprev;
    }
    if (cfg->edge_macro && !build_edge_points(s)) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

/* Set w and wdot; the distributions become f_eq(w, wdot), whose sum is wdot. */
void orc_set_fields(orc_state *s, const double *w, const double *wdot)
{
    size_t n = (size_t)s->c.nx * s->c.ny;
    for (size_t k = 0; k < n; ++k) {
        double feq[9];
        equilibrium_q(s, w[k], wdot[k], feq);
        s->w[k] = w[k];
        for (int a = 0; a < s->Q; ++a) s->f[a][k] = feq[a];
    }
}

/* w and wdot = sum_a f^a (eq. distrib-macro). */
void orc_get_fields(const orc_state *s, double *w, double *wdot)
{
    size_t n = (size_t)s->c.nx * s->c.ny;
    for (size_t k = 0; k < n; ++k) {
        double sum = 0.0;
        for (int a = 0; a < s->Q; ++a) sum += s->f[a][k];
        w[k] = s->w[k];
        wdot[k] = sum;
    }
}

void orc_get_distributions(const orc_state *s, double *f5)
{
    size_t n = (size_t)s->c.nx * s->c.ny;
    for (int a = 0; a < s->Q; ++a) memcpy(f5 + (size_t)a * n, s->f[a], n * sizeof(double));
}

void orc_get_cuts(const orc_state *s, uint8_t *cut_h, uint8_t *cut_v)
{
    size_t n = (size_t)s->c.nx * s->c.ny;
    memcpy(cut_h, s->cut_h, n);
    memcpy(cut_v, s->cut_v, n);
}

/* D2Q9: the severed flags of the diagonal links (i,j)-(i+1,j+1) and
 * (i+1,j)-(i,j+1), stored at (i,j). */
void orc_get_cuts_diag(const orc_state *s, uint8_t *cut_d1, uint8_t *cut_d2)
{
    size_t n = (size_t)s->c.nx * s->c.ny;
    memcpy(cut_d1, s->cut_d1, n);
    memcpy(cut_d2, s->cut_d2, n);
}

int32_t orc_q(const orc_state *s) { return s->Q; }

/* --------------------------------------------- macroscopic boundary points */

/* Bilinear interpolation stencil of the point (px, py) (units of dh, site
 * centres at half integers): up to four sites and weights. */
static int bilinear(const orc_state *s, double px, double py, int32_t idx[4], double wt[4])
{
    double gx = px - 0.5, gy = py - 0.5;
    int i0 = (int)floor(gx), j0 = (int)floor(gy);
    double tx = gx - i0, ty = gy - j0;
    int n = 0;
    for (int dj = 0; dj <= 1; ++dj)
        for (int di = 0; di <= 1; ++di) {
            double wgt = (di ? tx : 1.0 - tx) * (dj ? ty : 1.0 - ty);
            if (wgt == 0.0) continue;
            int i = i0 + di, j = j0 + dj;
            if (i < 0 || i >= s->c.nx || j < 0 || j >= s->c.ny) return -1;
            idx[n] = j * s->c.nx + i;
            wt[n] = wgt;
            ++n;
        }
    return n;
}

/* ProcessPoints for one new boundary point x_B (Sec. 3.1 and Alg. 1): the
 * closest point x_C on the crack, the normal through x_B, the interior points
 * x_I = x_B + dh n and x_II = x_B + 2 dh n with their bilinear stencils. */
/* ProcessPoints for a crack in any direction (the reading for a crack that
 * is not aligned with the lattice): x_B takes the normal n of the crack's
 * line, pointing away from it, so its stencil depends on the site and the
 * line alone; s_B is its distance from the line, and x_I = x_B + n dh,
 * x_II = x_B + 2 n dh.  Every corner of their bilinear cells is x_B plus a
 * step of the lattice in n's quadrant, so it lies at least as far from the
 * line as x_B, on its side: the stencils never reach across the crack. */
static void add_bpoint_line(orc_state *s, int32_t k, orc_bpoint *b)
{
    int nx = s->c.nx;
    double bx = k % nx + 0.5, by = k / nx + 0.5;
    double sx = (double)s->start_q / (double)qone(), sy = (double)s->start_yq / (double)qone();
    double d = -(bx - sx) * s->dir_y + (by - sy) * s->dir_x;
    double side = d > 0.0 ? 1.0 : -1.0;
    double nxv = -s->dir_y * side, nyv = s->dir_x * side;   /* away from the line */
    b->nI = bilinear(s, bx + nxv, by + nyv, b->idxI, b->wI);
    b->nII = bilinear(s, bx + 2.0 * nxv, by + 2.0 * nyv, b->idxII, b->wII);
    b->sB = fabs(d);
    b->sI = fabs(d) + 1.0;
    b->sII = fabs(d) + 2.0;
    if (b->nI < 0 || b->nII < 0) s->flags |= ORC_FLAG_UNSUPPORTED;
}

static void add_bpoint(orc_state *s, int32_t k)
{
    if (s->is_bpoint[k]) return;
    if (s->c.line) {
        if (s->nbl == s->capbl) {
            s->capbl *= 2;
            s->bl = realloc(s->bl, sizeof(orc_bpoint) * (size_t)s->capbl);
        }
        orc_bpoint *b = &s->bl[s->nbl];
        memset(b, 0, sizeof(*b));
        b->site = k;
        add_bpoint_line(s, k, b);
        s->is_bpoint[k] = 1;
        s->nbl++;
        return;
    }
    int nx = s->c.nx;
    int i = k % nx, j = k / nx;
    double bx = i + 0.5, by = j + 0.5;                   /* units of dh */
    double x0 = (double)(s->c.two_tips ? s->ltip_q : s->start_q) / (double)qone();
    double x1 = (double)s->tip_q / (double)qone();
    double yc = (double)s->c.jc;
    double cx = bx < x0 ? x0 : (bx > x1 ? x1 : bx);      /* closest point on the crack line segment */
    /* D2Q9: a site can lose only a diagonal link to the crack while its
     * centre lies beyond an end of the segment; its boundary condition is
     * that of the crack face the link crosses, whose normal is vertical */
    if (s->Q == 9) cx = bx;
    double cy = yc;
    double dx = bx - cx, dy = by - cy;
    double d = sqrt(dx * dx + dy * dy);
    if (s->nbl == s->capbl) {
        s->capbl *= 2;
        s->bl = realloc(s->bl, sizeof(orc_bpoint) * (size_t)s->capbl);
    }
    orc_bpoint *b = &s->bl[s->nbl];
    memset(b, 0, sizeof(*b));
    b->site = k;
    double nxv = dx / d, nyv = dy / d;
    b->sB = d;
    b->sI = d + 1.0;
    b->sII = d + 2.0;
    b->nI = bilinear(s, bx + nxv, by + nyv, b->idxI, b->wI);
    b->nII = bilinear(s, bx + 2.0 * nxv, by + 2.0 * nyv, b->idxII, b->wII);
    if (b->nI < 0 || b->nII < 0) s->flags |= ORC_FLAG_UNSUPPORTED;
    s->is_bpoint[k] = 1;
    s->nbl++;
}

/* w at x_B from the quadratic polynomial p(s) = a + b s^2 (zero normal
 * derivative on a traction-free face) through (s_I, w_I) and (s_II, w_II). */
static double macro_value(const orc_bpoint *b, const double *w)
{
    double wI = 0.0, wII = 0.0;
    for (int q = 0; q < b->nI; ++q) wI += b->wI[q] * w[b->idxI[q]];
    for (int q = 0; q < b->nII; ++q) wII += b->wII[q] * w[b->idxII[q]];
    double bb = (wII - wI) / (b->sII * b->sII - b->sI * b->sI);
    double aa = wI - bb * b->sI * b->sI;
    return aa + bb * b->sB * b->sB;
}

/* The same polynomial evaluated for given values (for the tests). */
double orc_macro_poly(double sB, double sI, double sII, double wI, double wII)
{
    orc_bpoint b;
    double w[2] = {wI, wII};
    memset(&b, 0, sizeof b);
    b.nI = 1; b.idxI[0] = 0; b.wI[0] = 1.0;
    b.nII = 1; b.idxII[0] = 1; b.wII[0] = 1.0;
    b.sB = sB; b.sI = sI; b.sII = sII;
    return macro_value(&b, w);
}

/* The quadratic polynomial through (s0, v0), (s1, v1), (s2, v2), evaluated
 * at x (Lagrange form).  On a Dirichlet edge (Sec. 3.1) the three points are
 * the boundary value at the edge and w at x_I and x_II. */
static double quadratic_through(double s0, double v0, double s1, double v1, double s2, double v2, double x)
{
    return v0 * (x - s1) * (x - s2) / ((s0 - s1) * (s0 - s2))
         + v1 * (x - s0) * (x - s2) / ((s1 - s0) * (s1 - s2))
         + v2 * (x - s0) * (x - s1) / ((s2 - s0) * (s2 - s1));
}

double orc_quadratic_through(double s0, double v0, double s1, double v1, double s2, double v2, double x)
{
    return quadratic_through(s0, v0, s1, v1, s2, v2, x);
}

/* The outer-edge boundary points of the macroscopic rule (Sec. 3.1): every
 * site next to a free or Dirichlet edge.  The outer edges lie half a spacing
 * outside the edge sites, so along the inward normal x_B, x_I, x_II sit at
 * the distances 1/2, 3/2, 5/2 dh from the edge and x_I, x_II are lattice
 * sites (their bilinear interpolation is the site value).  A corner between
 * two such edges follows the Dirichlet one; when both are of one kind it
 * follows the bottom or top edge.  Returns 0 where the rule is not defined:
 * fewer than four sites across a pair of edges (x_II would be a boundary
 * point of the opposite edge), or a crack within four rows of the bottom or
 * top edge (a crack face point's x_II would lie on the edge). */
static int build_edge_points(orc_state *s)
{
    const orc_config *c = &s->c;
    int nx = c->nx, ny = c->ny;
    int onL = c->edge[ORC_LEFT] != ORC_PERIODIC, onR = c->edge[ORC_RIGHT] != ORC_PERIODIC;
    int onB = c->edge[ORC_BOTTOM] != ORC_PERIODIC, onT = c->edge[ORC_TOP] != ORC_PERIODIC;
    if ((onL || onR) && nx < 4) return 0;
    if ((onB || onT) && ny < 4) return 0;
    if (c->crack_mode != ORC_CRACK_NONE && (c->jc < 4 || c->jc > ny - 4)) return 0;
    static const int NX_[4] = {1, -1, 0, 0}, NY_[4] = {0, 0, 1, -1};   /* inward normals */
    s->ep = xcalloc((size_t)2 * ((size_t)nx + ny), sizeof(orc_epoint));
    s->nep = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int eh = (onL && i == 0) ? ORC_LEFT : (onR && i == nx - 1) ? ORC_RIGHT : -1;
            int ev = (onB && j == 0) ? ORC_BOTTOM : (onT && j == ny - 1) ? ORC_TOP : -1;
            if (eh < 0 && ev < 0) continue;
            int e;
            if (eh >= 0 && ev >= 0)
                e = (c->edge[eh] == ORC_DIRICHLET && c->edge[ev] != ORC_DIRICHLET) ? eh : ev;
            else
                e = ev >= 0 ? ev : eh;
            orc_epoint *p = &s->ep[s->nep++];
            p->site = j * nx + i;
            p->I = (j + NY_[e]) * nx + (i + NX_[e]);
            p->II = (j + 2 * NY_[e]) * nx + (i + 2 * NX_[e]);
            p->edge = e;
            p->rule = c->edge[e] == ORC_DIRICHLET;
        }
    return 1;
}

/* w_B of an outer-edge point from the quadratic along its normal, with the
 * distances from the edge in units of dh: traction free, the polynomial
 * a + b s^2 (zero normal derivative at the edge) through x_I and x_II;
 * Dirichlet, the polynomial through (0, w*), x_I and x_II. */
static double edge_value(const orc_epoint *p, const double *w, const double *wstar)
{
    const double sB = 0.5, sI = 1.5, sII = 2.5;
    if (p->rule) return quadratic_through(0.0, wstar[p->edge], sI, w[p->I], sII, w[p->II], sB);
    return orc_macro_poly(sB, sI, sII, w[p->I], w[p->II]);
}

/* eq. f-macro-bc: the distributions that site k misses (links leaving the
 * domain or severed) share equally what makes sum_a f^a = (w_B - w(t)) / dt. */
static void set_missing(orc_state *s, int32_t k, double wB)
{
    int miss[8], nmiss = 0;
    double known = s->f[0][k];
    for (int a = 1; a < s->Q; ++a) {
        uint8_t *cut;
        int32_t src = link_of(s, k, OPP[a], &cut);
        if (src < 0 || *cut) miss[nmiss++] = a;
        else known += s->f[a][k];
    }
    double target = (wB - s->w_old[k]) / s->c.dt;
    for (int q = 0; q < nmiss; ++q) s->f[miss[q]][k] = (target - known) / (double)nmiss;
    s->w[k] = wB;
}

/* The macroscopic rule (Sec. 3.1): solve S(t+dt) w_B(t+dt) = R(t+dt) for
 * the boundary points of the crack faces and, if enabled, the outer edges,
 * then set their missing distributions by eq. f-macro-bc.  Each point's
 * equation reads w_B = polynomial(interior values), where an interior value
 * may itself be a boundary unknown (a corner reads edge points; a crack face
 * point on an edge column reads edge points).  Jacobi sweeps from the values
 * of the LBM update: a sweep that changes no bit has met every equation. */
static void boundary_solve(orc_state *s)
{
    int crack_rule = s->c.bc_mode == ORC_BC_MACROSCOPIC;
    int nb = crack_rule ? s->nbl : 0;
    int ne = s->c.edge_macro ? s->nep : 0;
    if (nb + ne == 0) return;
    size_t n = (size_t)s->c.nx * s->c.ny;
    double wstar[4];
    for (int e = 0; e < 4; ++e) wstar[e] = load_value(s, e, s->step + 1);   /* w*(t_n+1) */
    double *cur = malloc(sizeof(double) * n);
    double *val = malloc(sizeof(double) * (size_t)(nb + ne + 1));
    int32_t *site = malloc(sizeof(int32_t) * (size_t)(nb + ne + 1));
    int m = 0;
    for (int b = 0; b < nb; ++b) site[m++] = s->bl[b].site;
    for (int q = 0; q < ne; ++q)
        if (!(crack_rule && s->is_bpoint[s->ep[q].site])) site[m++] = s->ep[q].site;
    memcpy(cur, s->w, sizeof(double) * n);
    int converged = 0;
    for (int sweep = 0; sweep < 256 && !converged; ++sweep) {
        int v = 0;
        for (int b = 0; b < nb; ++b) val[v++] = macro_value(&s->bl[b], cur);
        for (int q = 0; q < ne; ++q)
            if (!(crack_rule && s->is_bpoint[s->ep[q].site])) val[v++] = edge_value(&s->ep[q], cur, wstar);
        converged = 1;
        for (int q = 0; q < m; ++q)
            if (memcmp(&val[q], &cur[site[q]], sizeof(double)) != 0) converged = 0;
        for (int q = 0; q < m; ++q) cur[site[q]] = val[q];
    }
    if (!converged) s->flags |= ORC_FLAG_UNSUPPORTED;
    for (int q = 0; q < m; ++q) set_missing(s, site[q], cur[site[q]]);
    free(cur); free(val); free(site);
}

/* -------------------------------------------------------------- LBM step */

/* The LBM step in two parts: the collision, and the rest (streaming, moment,
 * integration, the macroscopic rule).  A lattice split into row slabs hands
 * its boundary rows' post-collision values to the neighbours in between. */
static void lbm_collide(orc_state *s)
{
    size_t n = (size_t)s->c.nx * s->c.ny;
    double om = s->c.omega;
    int nth = s->threads > 1 ? s->threads : 1;
    (void)nth;
    /* collision (eq. LBE, right-hand side) */
#pragma omp parallel for num_threads(nth) schedule(static) if (nth > 1)
    for (size_t k = 0; k < n; ++k) {
        double wdot = 0.0;
        for (int a = 0; a < s->Q; ++a) wdot += s->f[a][k];
        double feq[9];
        equilibrium_q(s, s->w[k], wdot, feq);
        for (int a = 0; a < s->Q; ++a) s->fs[a][k] = s->f[a][k] - om * (s->f[a][k] - feq[a]);
    }
}

static void lbm_stream_rest(orc_state *s);

static void lbm_step(orc_state *s)
{
    lbm_collide(s);
    lbm_stream_rest(s);
}

static void lbm_stream_rest(orc_state *s)
{
    int nx = s->c.nx, ny = s->c.ny;
    size_t n = (size_t)nx * ny;
    double g = s->g, dt = s->c.dt;
    double wstar[4];
    for (int e = 0; e < 4; ++e) wstar[e] = load_value(s, e, s->step);

    /* The per-site loops (the collision above, and below) touch only their
     * own site or read the post-collision values of other sites, so they may
     * run on several threads without changing any result; the thread count
     * is 1 unless orc_set_threads raised it (timing runs only). */
    int nth = s->threads > 1 ? s->threads : 1;
    (void)nth;
    /* streaming along intact links (eq. LBE, left-hand side); a missing link
     * takes bounce-back (free edge, crack face) or anti-bounce-back (Dirichlet) */
#pragma omp parallel for num_threads(nth) schedule(static) if (nth > 1)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int32_t k = j * nx + i;
            s->f[0][k] = s->fs[0][k];
            for (int a = 1; a < s->Q; ++a) {
                int b = OPP[a];
                uint8_t *cut;
                int32_t src = link_of(s, k, b, &cut);     /* f^a arrives from x - c^a */
                if (src >= 0 && !*cut) {
                    s->f[a][k] = s->fs[a][src];
                } else if (src < 0) {
                    int e = missing_edge(s, k, b);
                    if (s->c.edge[e] == ORC_DIRICHLET)
                        s->f[a][k] = -s->fs[b][k] + 2.0 * weight(s, a) * g * wstar[e];
                    else if (s->c.edge[e] == ORC_HALO) {   /* from the neighbouring slab */
                        /* its source site's column in the neighbour's boundary
                         * row (across a periodic left / right edge, wrapped) */
                        int si = i - CX[a];
                        if (si < 0 || si >= nx) si = (si + nx) % nx;
                        s->f[a][k] = s->halo[e == ORC_BOTTOM ? 0 : 1][halo_slot(a)][si];
                    }
                    else
                        s->f[a][k] = s->fs[b][k];
                } else {
                    s->f[a][k] = s->fs[b][k];
                }
            }
        }
    /* moment and Euler integration (eqs. distrib-macro, integration) */
    memcpy(s->w_old, s->w, n * sizeof(double));
#pragma omp parallel for num_threads(nth) schedule(static) if (nth > 1)
    for (size_t k = 0; k < n; ++k) {
        double wdot = 0.0;
        for (int a = 0; a < s->Q; ++a) wdot += s->f[a][k];
        s->w[k] = s->w_old[k] + dt * wdot;
    }
    /* the macroscopic non-lattice-conforming rule on the boundary points */
    boundary_solve(s);
    s->step += 1;
}

/* --------------------------------------------------------- crack handling */

/* K from the crack opening of the site pairs (i, jc-1) / (i, jc) whose
 * distance r = tip - (i + 1/2) dh along the crack lies in [r_min, r_min + W)
 * (Sec. 4.2): least squares of delta_i = (4K/mu) s_i, s_i = sqrt(r_i / 2pi)
 * (eq. sif).  With one pair this is K = delta (mu/4) sqrt(2pi/r). */
static double evaluate_K_dir(const orc_state *s, const double *w, int64_t tip_q, double r_min, double wfit,
                             int dir, int32_t *npairs)
{
    int nx = s->c.nx, jc = s->c.jc;
    double dh = s->c.dh;
    double num = 0.0, den = 0.0;
    int np = 0;
    double lo = r_min / dh, hi = (r_min + wfit) / dh;
    for (int i = 0; i < nx; ++i) {
        if (!s->cut_v[(jc - 1) * nx + i]) continue;       /* the pair must straddle the crack */
        /* r along the crack behind the tip: tip - x_i for the right tip, x_i - tip for the left */
        double r_h = (double)(dir > 0 ? tip_q - site_cx_q(i) : site_cx_q(i) - tip_q) / (double)qone();
        if (!(r_h >= lo && r_h < hi)) continue;
        double r = r_h * dh;
        double sfac = sqrt(r / (2.0 * ORC_PI));
        double delta = w[jc * nx + i] - w[(jc - 1) * nx + i];
        num += delta * sfac;
        den += sfac * sfac;
        ++np;
    }
    *npairs = np;
    if (np == 0) return 0.0;
    return s->c.mu / 4.0 * num / den;
}

/* K at the tip (tx, ty) of a crack in any direction (Sec. 4.2 read for a
 * crack that is not aligned with the lattice): the pairs of sites adjacent
 * to the crack are the two ends of each severed link; the pair's distance
 * from the tip along the crack is that of the link's midpoint m,
 * r = (x_tip - m) . c (c the unit direction of growth; r = (m - x_tip) . c
 * at the left end of a two-tip crack, dir = -1), and the opening is
 * delta = w(left of c) - w(right of c) at both ends, so that a crack along
 * +x has the pairs, distances and opening of evaluate_K_dir.  The
 * projection is formed without fused multiply-adds, as in line_setup. */
static double evaluate_K_line(const orc_state *s, const double *w, int64_t tx, int64_t ty, double r_min, double wfit,
                              int dir, int32_t *npairs)
{
    int nx = s->c.nx, ny = s->c.ny;
    double dh = s->c.dh;
    double num = 0.0, den = 0.0;
    int np = 0;
    double lo = r_min / dh, hi = (r_min + wfit) / dh;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            for (int vert = 0; vert <= 1; ++vert) {
                int32_t k0 = j * nx + i, k1;
                int64_t mx, my;
                if (!vert) {
                    if (i + 1 >= nx || !s->cut_h[k0]) continue;
                    k1 = k0 + 1;
                    mx = (int64_t)(i + 1) << ORC_Q;
                    my = site_cx_q(j);
                } else {
                    if (j + 1 >= ny || !s->cut_v[k0]) continue;
                    k1 = k0 + nx;
                    mx = site_cx_q(i);
                    my = (int64_t)(j + 1) << ORC_Q;
                }
                /* behind the tip: along -c from the right end, along +c from the left end */
                volatile double px = (double)(dir > 0 ? tx - mx : mx - tx) / (double)qone() * s->dir_x;
                volatile double py = (double)(dir > 0 ? ty - my : my - ty) / (double)qone() * s->dir_y;
                double r_h = px + py;
                if (!(r_h >= lo && r_h < hi)) continue;
                /* k1 is the site at +x (horizontal link) or +y (vertical
                 * link); it lies left of c when c_y < 0, resp. c_x > 0 */
                int k1_left = vert ? s->dir_x > 0.0 : s->dir_y < 0.0;
                double delta = k1_left ? w[k1] - w[k0] : w[k0] - w[k1];
                double r = r_h * dh;
                double sfac = sqrt(r / (2.0 * ORC_PI));
                num += delta * sfac;
                den += sfac * sfac;
                ++np;
            }
    *npairs = np;
    if (np == 0) return 0.0;
    return s->c.mu / 4.0 * num / den;
}

double orc_evaluate_K_line(const orc_state *s, const double *w, int64_t tx, int64_t ty, double r_min, double wfit,
                           int32_t *npairs)
{
    return evaluate_K_line(s, w, tx, ty, r_min, wfit, +1, npairs);
}

static double evaluate_K(const orc_state *s, const double *w, int64_t tip_q, double r_min, double wfit, int32_t *npairs)
{
    return evaluate_K_dir(s, w, tip_q, r_min, wfit, +1, npairs);
}

double orc_evaluate_K(const orc_state *s, const double *w, int64_t tip_q, double r_min, double wfit, int32_t *npairs)
{
    return evaluate_K(s, w, tip_q, r_min, wfit, npairs);
}

/* K at a left tip (a crack end growing towards -x): the pairs at r = x_i - tip
 * in the window, the same opening delta = w(above) - w(below), so that a
 * mirror-symmetric problem has the same K at both ends. */
double orc_evaluate_K_left(const orc_state *s, const double *w, int64_t tip_q, double r_min, double wfit, int32_t *npairs)
{
    return evaluate_K_dir(s, w, tip_q, r_min, wfit, -1, npairs);
}

/* Alg. 1, CheckLinks: breadth-first search from the neighbours of the
 * previous boundary points.  A popped point p is marked visited, each intact
 * link (p, n_p) is tested against the new crack segment; an intersected link
 * puts both end points into B and the unvisited neighbours of n_p into the
 * queue.  The links found are severed after the search. */
static int checklinks(orc_state *s, int64_t ax, int64_t ay, int64_t bx, int64_t by, int32_t *B, int nBmax)
{
    int nx = s->c.nx;
    size_t n = (size_t)nx * s->c.ny;
    int32_t qh = 0, qt = 0;
    int nB = 0;
    uint8_t *tocut[4096];
    int ncut = 0;
    memset(s->inq, 0, n);
    memset(s->visited, 0, n);
    for (int b = 0; b < s->nbprev; ++b)
        for (int a = 1; a < s->Q; ++a) {
            uint8_t *cut;
            int32_t m = link_of(s, s->bprev[b], a, &cut);
            if (m >= 0 && !*cut && !s->inq[m]) { s->inq[m] = 1; s->queue[qt++] = m; }
        }
    if (s->nbprev == 0) {
        /* no previous boundary points: start from the sites around the old tip */
        int64_t half = qone() / 2;
        int i0 = (int)((ax - half) >> ORC_Q), j0 = (int)((ay - half) >> ORC_Q);   /* floor(x/dh - 1/2) */
        for (int j = j0; j <= j0 + 1; ++j)
            for (int i = i0; i <= i0 + 1; ++i)
                if (i >= 0 && i < nx && j >= 0 && j < s->c.ny && !s->inq[j * nx + i]) {
                    s->inq[j * nx + i] = 1;
                    s->queue[qt++] = j * nx + i;
                }
    }
    while (qh < qt) {
        int32_t p = s->queue[qh++];
        s->visited[p] = 1;
        int pi = p % nx, pj = p / nx;
        for (int a = 1; a < s->Q; ++a) {
            uint8_t *cut;
            int wrap;
            int32_t m = link_of_w(s, p, a, &cut, &wrap);
            if (m < 0 || *cut || wrap) continue;   /* a link across a periodic edge lies outside the body */
            int mi = m % nx, mj = m / nx;
            if (!orc_segments_intersect(site_cx_q(pi), site_cx_q(pj), site_cx_q(mi), site_cx_q(mj), ax, ay, bx, by))
                continue;
            int seen = 0;
            for (int q = 0; q < ncut; ++q) seen |= tocut[q] == cut;
            if (!seen && ncut < 4096) tocut[ncut++] = cut;
            int hp = 0, hm = 0;
            for (int q = 0; q < nB; ++q) { hp |= B[q] == p; hm |= B[q] == m; }
            if (!hp && nB < nBmax) B[nB++] = p;
            if (!hm && nB < nBmax) B[nB++] = m;
            for (int c2 = 1; c2 < s->Q; ++c2) {
                uint8_t *cut2;
                int32_t r = link_of(s, m, c2, &cut2);
                if (r >= 0 && !*cut2 && !s->visited[r] && !s->inq[r]) { s->inq[r] = 1; s->queue[qt++] = r; }
            }
        }
    }
    for (int q = 0; q < ncut; ++q) *tocut[q] = 1;
    return nB;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* The criterion of Alg. 1 for one tip (dir = +1: the right end, growing
 * towards +x; -1: the left end of a two-tip crack, growing towards -x):
 * r_min of eq. r(v) from that tip's previous speed, K (eq. sif), and the
 * decision: prescribed growth, or |K| > K_C with the speed of eq. v-tanh. */
static void tip_criterion(const orc_state *s, int dir, double v_prev, int64_t tip, double *K, double *v, int *propagate,
                          int32_t *np)
{
    const orc_config *c = &s->c;
    double r_min = c->r_min_fixed > 0.0 ? c->r_min_fixed : c->r0 / (1.0 - v_prev);  /* eq. r(v) */
    *K = c->line ? evaluate_K_line(s, s->w, tip, dir > 0 ? s->tip_yq : s->ltip_yq, r_min, c->fit_width, dir, np)
                 : evaluate_K_dir(s, s->w, tip, r_min, c->fit_width, dir, np);
    *propagate = 0;
    *v = 0.0;
    if (c->crack_mode == ORC_CRACK_PRESCRIBED) {
        *propagate = 1;
        *v = c->v_rel;
    } else if (c->crack_mode == ORC_CRACK_KCRIT && *np > 0 && fabs(*K) > c->K_C) {
        double ratio = fabs(*K) / c->K_C;
        *propagate = 1;
        *v = c->v_max * tanh(sqrt(ratio * ratio * ratio * ratio - 1.0));  /* eq. v-tanh */
    }
}

/* A tip of a crack in any direction that would reach or cross the boundary
 * of the body [0, nx dh] x [0, ny dh] stops on it, where the segment from
 * the old tip (px, py) to (*qx, *qy) meets it first; the point is formed
 * in exact integer arithmetic (the quotient truncated towards zero).
 * Returns 1 if the tip was stopped. */
static int line_clamp(const orc_state *s, int64_t px, int64_t py, int64_t *qx, int64_t *qy)
{
    int64_t X = (int64_t)s->c.nx << ORC_Q, Y = (int64_t)s->c.ny << ORC_Q;
    int64_t dx = *qx - px, dy = *qy - py;
    int hitx = (dx > 0 && *qx >= X) || (dx < 0 && *qx <= 0);
    int hity = (dy > 0 && *qy >= Y) || (dy < 0 && *qy <= 0);
    if (!hitx && !hity) return 0;
    int64_t fx = dx > 0 ? X : 0, fy = dy > 0 ? Y : 0;
    __int128 ux = (__int128)(fx - px), uy = (__int128)(fy - py);
    int xfirst = hitx;
    if (hitx && hity) {
        /* the face met first: t_x = ux / dx against t_y = uy / dy, both in [0, 1] */
        __int128 ax = ux < 0 ? -ux : ux, ay = uy < 0 ? -uy : uy;
        __int128 adx = dx < 0 ? -(__int128)dx : dx, ady = dy < 0 ? -(__int128)dy : dy;
        xfirst = ax * ady <= ay * adx;
    }
    if (xfirst) {
        *qx = fx;
        *qy = py + (int64_t)(ux * dy / dx);
    } else {
        *qy = fy;
        *qx = px + (int64_t)(uy * dx / dy);
    }
    return 1;
}

/* Advance one tip by Delta a = adot dt (towards +x or -x, stopping at the far
 * edge), sever the links the new segment intersects (CheckLinks from that
 * tip's previous boundary points) and register the new boundary points
 * (ProcessPoints).  Returns 1 if the tip moved. */
static int tip_advance(orc_state *s, int dir, double v)
{
    const orc_config *c = &s->c;
    double adot = v * s->cs;
    int64_t dq = llrint(adot * c->dt / c->dh * (double)qone());   /* Delta a = adot dt */
    int64_t yq = (int64_t)c->jc << ORC_Q;
    int32_t B[64];
    int nB;
    if (c->line) {
        /* along the crack's direction (+c for the right end, -c for the
         * left one): each component of Delta a c rounded to the grid
         * (c = (1, 0) gives the advance below) */
        double q = adot * c->dt / c->dh * (double)qone();
        int64_t px = dir > 0 ? s->tip_q : s->ltip_q, py = dir > 0 ? s->tip_yq : s->ltip_yq;
        int64_t ax = llrint(q * s->dir_x), ay = llrint(q * s->dir_y);
        int64_t nxq = dir > 0 ? px + ax : px - ax, nyq = dir > 0 ? py + ay : py - ay;
        if (line_clamp(s, px, py, &nxq, &nyq)) {
            if (dir > 0) s->arrested_for_good = 1;
            else s->larrested = 1;
            s->flags |= ORC_FLAG_CLAMPED;
        }
        if (nxq == px && nyq == py) return 0;
        if (dir > 0) { s->tip_q = nxq; s->tip_yq = nyq; }
        else { s->ltip_q = nxq; s->ltip_yq = nyq; }
        int32_t *keep = s->bprev, nkeep = s->nbprev;   /* CheckLinks from this end's B_prev */
        if (dir < 0) { s->bprev = s->lbprev; s->nbprev = s->nlbprev; }
        nB = checklinks(s, px, py, nxq, nyq, B, 64);
        if (dir < 0) { s->bprev = keep; s->nbprev = nkeep; }
        qsort(B, (size_t)nB, sizeof(int32_t), cmp_i32);
        if (c->bc_mode == ORC_BC_MACROSCOPIC)
            for (int b = 0; b < nB; ++b) add_bpoint(s, B[b]);   /* ProcessPoints */
        if (nB > 0) {
            if (dir > 0) { memcpy(s->bprev, B, sizeof(int32_t) * (size_t)nB); s->nbprev = nB; }
            else { memcpy(s->lbprev, B, sizeof(int32_t) * (size_t)nB); s->nlbprev = nB; }
        }
        return 1;
    }
    if (dir > 0) {
        int64_t prev = s->tip_q, next = prev + dq;
        if (next >= s->clamp_q) { next = s->clamp_q; s->arrested_for_good = 1; s->flags |= ORC_FLAG_CLAMPED; }
        if (next <= prev) return 0;
        s->tip_q = next;
        nB = checklinks(s, prev, yq, next, yq, B, 64);
        qsort(B, (size_t)nB, sizeof(int32_t), cmp_i32);
        for (int b = 0; b < nB; ++b) add_bpoint(s, B[b]);        /* ProcessPoints */
        if (nB > 0) { memcpy(s->bprev, B, sizeof(int32_t) * (size_t)nB); s->nbprev = nB; }
    } else {
        int64_t prev = s->ltip_q, next = prev - dq;
        if (next <= 0) { next = 0; s->larrested = 1; s->flags |= ORC_FLAG_CLAMPED; }
        if (next >= prev) return 0;
        s->ltip_q = next;
        int32_t *keep = s->bprev, nkeep = s->nbprev;                /* CheckLinks from this tip's B_prev */
        s->bprev = s->lbprev;
        s->nbprev = s->nlbprev;
        nB = checklinks(s, prev, yq, next, yq, B, 64);
        s->bprev = keep;
        s->nbprev = nkeep;
        qsort(B, (size_t)nB, sizeof(int32_t), cmp_i32);
        for (int b = 0; b < nB; ++b) add_bpoint(s, B[b]);
        if (nB > 0) { memcpy(s->lbprev, B, sizeof(int32_t) * (size_t)nB); s->nlbprev = nB; }
    }
    return 1;
}

/* Alg. 1, CrackGrowth, appended after the LBM step (Sec. 4.1).  With two
 * tips both criteria are evaluated on the same state, then the right tip
 * and the left tip advance in that order. */
static void crack_growth(orc_state *s)
{
    const orc_config *c = &s->c;
    if (c->crack_mode == ORC_CRACK_NONE) return;
    double K, v, Kl = 0.0, vl = 0.0;
    int propagate, propl = 0;
    int32_t np, npl = 0;
    tip_criterion(s, +1, s->v_prev, s->tip_q, &K, &v, &propagate, &np);
    if (c->two_tips) tip_criterion(s, -1, s->lv_prev, s->ltip_q, &Kl, &vl, &propl, &npl);
    if (!isfinite(K) || !isfinite(Kl)) s->flags |= ORC_FLAG_NONFINITE;
    if (s->arrested_for_good) { propagate = 0; v = 0.0; }
    if (s->larrested) { propl = 0; vl = 0.0; }
    int grew = propagate ? tip_advance(s, +1, v) : 0;
    int grewl = (c->two_tips && propl) ? tip_advance(s, -1, vl) : 0;
    s->v_prev = c->crack_mode == ORC_CRACK_PRESCRIBED ? c->v_rel : v;
    s->K_last = K;
    s->npairs_last = np;
    if (c->two_tips) {
        s->lv_prev = c->crack_mode == ORC_CRACK_PRESCRIBED ? c->v_rel : vl;
        s->lK_last = Kl;
        s->lnpairs_last = npl;
    }
    if (s->hist_n < c->hist_cap) {
        int64_t h = s->hist_n;
        s->hK[h] = K; s->hv[h] = v; s->htip[h] = s->tip_q; s->hnp[h] = np; s->hgrow[h] = grew;
        s->hKl[h] = Kl; s->hvl[h] = vl; s->htipl[h] = s->ltip_q; s->hnpl[h] = npl; s->hgrowl[h] = grewl;
        s->htipy[h] = s->tip_yq;
        s->htipyl[h] = s->ltip_yq;
    }
    s->hist_n += 1;
}

/* Row slabs: orc_collide runs the collision of the next step; orc_fs_row
 * copies the post-collision values that leave the slab across its bottom
 * (side 0: f*^4, then f*^7, f*^8 with D2Q9, of row 0) or top (side 1: f*^2,
 * then f*^5, f*^6, of row ny-1) edge, orc_halo_width rows of nx; the
 * neighbour hands them to orc_set_halo (side 0: they arrive at row 0 as f^2,
 * f^5, f^6; side 1: at row ny-1 as f^4, f^7, f^8), each read at its link's
 * source column; orc_finish_step completes the step (streaming
 * and the rest, then the crack handling of Alg. 1).  orc_collide followed by
 * orc_finish_step is orc_step(s, 1). */
void orc_collide(orc_state *s) { lbm_collide(s); }

/* Values per column of a boundary row handed over: 1 (D2Q5) or 3 (D2Q9). */
int32_t orc_halo_width(const orc_state *s) { return s->Q == 9 ? 3 : 1; }

void orc_fs_row(const orc_state *s, int32_t side, double *out)
{
    int nx = s->c.nx, nw = s->Q == 9 ? 3 : 1;
    size_t row = side == 0 ? 0 : (size_t)(s->c.ny - 1) * nx;
    for (int d = 0; d < nw; ++d) {
        const double *fs = s->fs[side == 0 ? HALO_DOWN[d] : HALO_UP[d]];
        for (int i = 0; i < nx; ++i) out[(size_t)d * nx + i] = fs[row + i];
    }
}

void orc_set_halo(orc_state *s, int32_t side, const double *in)
{
    int nx = s->c.nx, nw = s->Q == 9 ? 3 : 1;
    for (int d = 0; d < nw; ++d)
        for (int i = 0; i < nx; ++i) s->halo[side == 0 ? 0 : 1][d][i] = in[(size_t)d * nx + i];
}

void orc_finish_step(orc_state *s)
{
    lbm_stream_rest(s);
    crack_growth(s);
}

/* Threads for the per-site loops of the LBM step (timing of the CPU baseline;
 * results do not depend on it).  Returns the count in force: 1 when the
 * library was built without OpenMP. */
int32_t orc_set_threads(orc_state *s, int32_t n)
{
#ifdef _OPENMP
    s->threads = n > 1 ? n : 1;
#else
    (void)n;
    s->threads = 1;
#endif
    return s->threads;
}

/* Advance n time steps: the LBM step including its boundary rules, then the
 * crack handling (Sec. 4.1: appended at the end of each step). */
void orc_step(orc_state *s, int64_t n)
{
    for (int64_t q = 0; q < n; ++q) {
        lbm_step(s);
        crack_growth(s);
    }
}

/* ------------------------------------------------------------- inspection */

typedef struct {
    int64_t step, tip_q, hist_n;
    double K, v_prev;
    int32_t npairs, flags, n_bpoints, pad;
} orc_crack_info;

void orc_get_crack(const orc_state *s, orc_crack_info *out)
{
    out->step = s->step;
    out->tip_q = s->tip_q;
    out->hist_n = s->hist_n;
    out->K = s->K_last;
    out->v_prev = s->v_prev;
    out->npairs = s->npairs_last;
    out->flags = s->flags;
    out->n_bpoints = s->nbl;
    out->pad = 0;
}

int64_t orc_get_history(const orc_state *s, double *K, double *v, int64_t *tip_q, int32_t *npairs, int32_t *grew, int64_t cap)
{
    int64_t n = s->hist_n < s->c.hist_cap ? s->hist_n : s->c.hist_cap;
    if (n > cap) n = cap;
    for (int64_t h = 0; h < n; ++h) {
        K[h] = s->hK[h]; v[h] = s->hv[h]; tip_q[h] = s->htip[h]; npairs[h] = s->hnp[h]; grew[h] = s->hgrow[h];
    }
    return n;
}

int64_t orc_get_history_left(const orc_state *s, double *K, double *v, int64_t *tip_q, int32_t *npairs, int32_t *grew,
                             int64_t cap)
{
    int64_t n = s->hist_n < s->c.hist_cap ? s->hist_n : s->c.hist_cap;
    if (n > cap) n = cap;
    for (int64_t h = 0; h < n; ++h) {
        K[h] = s->hKl[h]; v[h] = s->hvl[h]; tip_q[h] = s->htipl[h]; npairs[h] = s->hnpl[h]; grew[h] = s->hgrowl[h];
    }
    return n;
}

int64_t orc_left_tip(const orc_state *s) { return s->ltip_q; }

/* The tip's y (units of 2^-32 dh) now and per step (crack in any direction). */
int64_t orc_tip_y(const orc_state *s) { return s->tip_yq; }
int64_t orc_get_history_y(const orc_state *s, int64_t *tip_yq, int64_t cap)
{
    int64_t n = s->hist_n < s->c.hist_cap ? s->hist_n : s->c.hist_cap;
    if (n > cap) n = cap;
    for (int64_t h = 0; h < n; ++h) tip_yq[h] = s->htipy[h];
    return n;
}
int64_t orc_left_tip_y(const orc_state *s) { return s->ltip_yq; }
int64_t orc_get_history_left_y(const orc_state *s, int64_t *tip_yq, int64_t cap)
{
    int64_t n = s->hist_n < s->c.hist_cap ? s->hist_n : s->c.hist_cap;
    if (n > cap) n = cap;
    for (int64_t h = 0; h < n; ++h) tip_yq[h] = s->htipyl[h];
    return n;
}
void orc_direction(const orc_state *s, double *dir2)
{
    dir2[0] = s->dir_x;
    dir2[1] = s->dir_y;
}

/* The outer-edge boundary points: site, x_I, x_II, rule and edge of each. */
int32_t orc_get_edge_points(const orc_state *s, int32_t *out5, int32_t cap)
{
    int32_t n = 0;
    for (int q = 0; q < s->nep && n < cap; ++q, ++n) {
        out5[5 * n + 0] = s->ep[q].site;
        out5[5 * n + 1] = s->ep[q].I;
        out5[5 * n + 2] = s->ep[q].II;
        out5[5 * n + 3] = s->ep[q].rule;
        out5[5 * n + 4] = s->ep[q].edge;
    }
    return s->nep;
}

int32_t orc_get_bpoints(const orc_state *s, int32_t *sites, int32_t cap)
{
    int32_t n = s->nbl < cap ? s->nbl : cap;
    for (int32_t b = 0; b < n; ++b) sites[b] = s->bl[b].site;
    return n;
}

/* Stand-alone CheckLinks on a lattice with the given severed links and
 * previous boundary points (for the brute-force comparison tests).  The cut
 * arrays are updated in place; returns the number of new boundary points. */
int32_t orc_checklinks_standalone(int32_t nx, int32_t ny, uint8_t *cut_h, uint8_t *cut_v,
                                  const int32_t *bprev, int32_t nbprev,
                                  int64_t ax, int64_t ay, int64_t bx, int64_t by,
                                  int32_t *B, int32_t nBmax)
{
    orc_state s;
    memset(&s, 0, sizeof s);
    s.c.nx = nx;
    s.c.ny = ny;
    s.Q = 5;
    s.cut_h = cut_h;
    s.cut_v = cut_v;
    size_t n = (size_t)nx * ny;
    s.queue = calloc(8 * n + 8, sizeof(int32_t));
    s.inq = calloc(n, 1);
    s.visited = calloc(n, 1);
    s.bprev = (int32_t *)bprev;
    s.nbprev = nbprev;
    int nB = checklinks(&s, ax, ay, bx, by, B, nBmax);
    free(s.queue); free(s.inq); free(s.visited);
    return nB;
}

double orc_load_value(const orc_state *s, int32_t edge, int64_t n) { return load_value(s, edge, n); }
double orc_g(const orc_state *s) { return s->g; }
int32_t orc_abi_version(void) { return 1; }

/* ------------------------------------------------------------ adjoint
 *
 * Gradient of the sensor misfit
 *     L = sum_{n=1..T} sum_s (w^n(x_s) - wbar^n_s)^2
 * with respect to the Dirichlet edge values w*_e(t_n) (n = 0..T-1), the
 * initial displacement w^0 and the initial rate wdot^0, with the crack's
 * cut schedule of the forward run held fixed (the crack decisions of Alg. 1
 * are discrete).  Under a fixed schedule one step of Sec. 3 is affine in the
 * state, so the gradient is the transpose of each step applied in reverse
 * order.  The transpose below is taken operation by operation from lbm_step
 * above (collision, streaming with bounce-back / anti-bounce-back,
 * eqs. distrib-macro and integration, and the macroscopic rule of Sec. 3.1),
 * on the oracle's own state (w, f^0..f^4). */

typedef struct {
    int32_t *ch, *cv;      /* step from which each link is severed (INT32_MAX: never) */
    int32_t *nbl;          /* boundary points in force during each step */
} orc_schedule;

/* Cut flags in force during step n. */
static void schedule_cuts(const orc_schedule *sc, size_t n_sites, int64_t n, uint8_t *cut_h, uint8_t *cut_v)
{
    for (size_t k = 0; k < n_sites; ++k) {
        cut_h[k] = sc->ch[k] <= n;
        cut_v[k] = sc->cv[k] <= n;
    }
}

/* Transpose of lbm_step for step n, given the adjoint (lw, lf) of the state
 * after the step; overwrites them with the adjoint of the state before it and
 * adds dL/dw*_e(t_n) to dload[e] (if dload is not NULL).  s->cut_h, s->cut_v
 * and the first nbl boundary points must be those in force during step n. */
static void lbm_step_transpose(orc_state *s, int nbl, double *lw, double *lf[5], double *dload4)
{
    int nx = s->c.nx, ny = s->c.ny;
    size_t n = (size_t)nx * ny;
    double g = s->g, om = s->c.omega, dt = s->c.dt;
    double *lw5 = malloc(sizeof(double) * n), *lwold = calloc(n, sizeof(double));
    double *lf4[5], *lfs[5];
    for (int a = 0; a < 5; ++a) {
        lf4[a] = malloc(sizeof(double) * n);
        lfs[a] = calloc(n, sizeof(double));
        memcpy(lf4[a], lf[a], sizeof(double) * n);
    }
    memcpy(lw5, lw, sizeof(double) * n);

    /* macroscopic rule: w(x_B) = p(s_B) from w at the stencils of x_I, x_II;
     * the missing f at x_B carry (target - known) / nmiss, target =
     * (w_B - w_old(x_B)) / dt */
    if (s->c.bc_mode == ORC_BC_MACROSCOPIC && nbl > 0) {
        double *lwB = calloc((size_t)nbl, sizeof(double));
        for (int b = 0; b < nbl; ++b) {
            int32_t k = s->bl[b].site;
            lwB[b] += lw[k];
            lw5[k] = 0.0;
            int miss[4], nmiss = 0;
            for (int a = 1; a < 5; ++a) {
                uint8_t *cut;
                int32_t src = link_of(s, k, OPP[a], &cut);
                if (src < 0 || *cut) miss[nmiss++] = a;
            }
            if (nmiss == 0) continue;
            /* sm is dL/dwdot at x_B after the step; it vanishes whenever x_B is
             * still a boundary point in the next step (wdot(x_B) is then
             * recomputed from w alone), i.e. always while the crack only grows.
             * The terms are kept as the literal transpose. */
            double sm = 0.0;
            for (int q = 0; q < nmiss; ++q) sm += lf[miss[q]][k];
            sm /= (double)nmiss;
            for (int a = 0; a < 5; ++a) {
                int is_miss = 0;
                for (int q = 0; q < nmiss; ++q) is_miss |= miss[q] == a;
                if (is_miss) lf4[a][k] = 0.0;
                else lf4[a][k] -= sm;
            }
            lwB[b] += sm / dt;
            lwold[k] -= sm / dt;
        }
        for (int b = 0; b < nbl; ++b) {
            const orc_bpoint *B = &s->bl[b];
            /* p(s_B) = (1 - r) w_I + r w_II, r = (s_B^2 - s_I^2) / (s_II^2 - s_I^2) */
            double r = (B->sB * B->sB - B->sI * B->sI) / (B->sII * B->sII - B->sI * B->sI);
            for (int q = 0; q < B->nI; ++q) lw5[B->idxI[q]] += (1.0 - r) * B->wI[q] * lwB[b];
            for (int q = 0; q < B->nII; ++q) lw5[B->idxII[q]] += r * B->wII[q] * lwB[b];
        }
        free(lwB);
    }
    /* w = w_old + dt sum_a f^a */
    for (size_t k = 0; k < n; ++k) {
        lwold[k] += lw5[k];
        for (int a = 0; a < 5; ++a) lf4[a][k] += dt * lw5[k];
    }
    /* streaming with the boundary rules */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int32_t k = j * nx + i;
            lfs[0][k] += lf4[0][k];
            for (int a = 1; a < 5; ++a) {
                int b = OPP[a];
                uint8_t *cut;
                int32_t src = link_of(s, k, b, &cut);
                if (src >= 0 && !*cut) {
                    lfs[a][src] += lf4[a][k];
                } else if (src < 0) {
                    int e = (b == 1) ? ORC_RIGHT : (b == 3) ? ORC_LEFT : (b == 2) ? ORC_TOP : ORC_BOTTOM;
                    if (s->c.edge[e] == ORC_DIRICHLET) {
                        lfs[b][k] -= lf4[a][k];
                        if (dload4) dload4[e] += 2.0 * g * lf4[a][k];
                    } else {
                        lfs[b][k] += lf4[a][k];
                    }
                } else {
                    lfs[b][k] += lf4[a][k];
                }
            }
        }
    /* collision f* = f - om (f - f_eq(w, wdot)), wdot = sum_a f^a */
    for (size_t k = 0; k < n; ++k) {
        double lfeq[5], lwdot;
        for (int a = 0; a < 5; ++a) lfeq[a] = om * lfs[a][k];
        lwdot = lfeq[0];
        double lwk = lwold[k] - 4.0 * g * lfeq[0];
        for (int a = 1; a < 5; ++a) lwk += g * lfeq[a];
        lw[k] = lwk;
        for (int a = 0; a < 5; ++a) lf[a][k] = (1.0 - om) * lfs[a][k] + lwdot;
    }
    for (int a = 0; a < 5; ++a) { free(lf4[a]); free(lfs[a]); }
    free(lw5);
    free(lwold);
}

/* Forward run of T steps from (w0, wdot0) with the sensor trace, the misfit L
 * and, if any of dload / dw0 / dwd0 is not NULL, its gradient by the
 * transposed steps.  Sensors are sites (si[k], sj[k]); target and trace are
 * T x ns (row n-1 holds state n).  dload is 4 x T (row e: dL/dw*_e(t_n),
 * zero for edges that are not Dirichlet).  Returns 0, or -1 for bad input. */
int orc_adjoint(const orc_config *cfg, const double *w0, const double *wd0, int64_t T, int32_t ns,
                const int32_t *si, const int32_t *sj, const double *target, double *loss, double *trace,
                double *dload, double *dw0, double *dwd0)
{
    /* the transposed step covers D2Q5 and the crack-face rule only, not the
     * macroscopic rule on the outer edges */
    if (T < 1 || ns < 0 || cfg->edge_macro || (cfg->q != 0 && cfg->q != 5)) return -1;
    orc_state *s = orc_create(cfg);
    if (!s) return -1;
    int nx = s->c.nx, ny = s->c.ny;
    size_t n = (size_t)nx * ny;
    for (int32_t k = 0; k < ns; ++k)
        if (si[k] < 0 || si[k] >= nx || sj[k] < 0 || sj[k] >= ny) { orc_destroy(s); return -1; }
    double *wz = calloc(n, sizeof(double));
    orc_set_fields(s, w0 ? w0 : wz, wd0 ? wd0 : wz);
    free(wz);

    orc_schedule sc;
    sc.ch = malloc(sizeof(int32_t) * n);
    sc.cv = malloc(sizeof(int32_t) * n);
    sc.nbl = malloc(sizeof(int32_t) * (size_t)T);
    for (size_t k = 0; k < n; ++k) {
        sc.ch[k] = s->cut_h[k] ? 0 : INT32_MAX;
        sc.cv[k] = s->cut_v[k] ? 0 : INT32_MAX;
    }
    double *res = malloc(sizeof(double) * (size_t)T * (size_t)(ns > 0 ? ns : 1));
    double L = 0.0;
    for (int64_t q = 0; q < T; ++q) {
        sc.nbl[q] = s->nbl;
        orc_step(s, 1);   /* LBM step q, then the crack step that fixes the cuts of step q + 1 */
        for (size_t k = 0; k < n; ++k) {
            if (s->cut_h[k] && sc.ch[k] == INT32_MAX) sc.ch[k] = (int32_t)(q + 1);
            if (s->cut_v[k] && sc.cv[k] == INT32_MAX) sc.cv[k] = (int32_t)(q + 1);
        }
        for (int32_t k = 0; k < ns; ++k) {
            double wk = s->w[(size_t)sj[k] * nx + si[k]];
            double r = wk - target[q * ns + k];
            if (trace) trace[q * ns + k] = wk;
            res[q * ns + k] = r;
            L += r * r;
        }
    }
    if (loss) *loss = L;

    if (dload || dw0 || dwd0) {
        double *lw = calloc(n, sizeof(double)), *lf[5];
        for (int a = 0; a < 5; ++a) lf[a] = calloc(n, sizeof(double));
        uint8_t *keep_h = s->cut_h, *keep_v = s->cut_v;
        uint8_t *ch = malloc(n), *cv = malloc(n);
        s->cut_h = ch;
        s->cut_v = cv;
        if (dload) memset(dload, 0, sizeof(double) * 4 * (size_t)T);
        /* dL/dw^T from the last state's misfit */
        for (int32_t k = 0; k < ns; ++k) lw[(size_t)sj[k] * nx + si[k]] += 2.0 * res[(T - 1) * ns + k];
        for (int64_t q = T - 1; q >= 0; --q) {
            double d4[4] = {0.0, 0.0, 0.0, 0.0};
            schedule_cuts(&sc, n, q, ch, cv);
            lbm_step_transpose(s, sc.nbl[q], lw, lf, d4);
            if (dload)
                for (int e = 0; e < 4; ++e) dload[(size_t)e * T + q] = d4[e];
            if (q >= 1)   /* misfit of state q */
                for (int32_t k = 0; k < ns; ++k) lw[(size_t)sj[k] * nx + si[k]] += 2.0 * res[(q - 1) * ns + k];
        }
        /* f = f_eq(w0, wdot0) at the start: f^0 = wdot0 - 4 g w0, f^k = g w0 */
        for (size_t k = 0; k < n; ++k) {
            if (dw0) dw0[k] = lw[k] - 4.0 * s->g * lf[0][k] + s->g * (lf[1][k] + lf[2][k] + lf[3][k] + lf[4][k]);
            if (dwd0) dwd0[k] = lf[0][k];
        }
        s->cut_h = keep_h;
        s->cut_v = keep_v;
        free(ch);
        free(cv);
        free(lw);
        for (int a = 0; a < 5; ++a) free(lf[a]);
    }
    free(res);
    free(sc.ch);
    free(sc.cv);
    free(sc.nbl);
    orc_destroy(s);
    return 0;
}
