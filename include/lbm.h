/*
 * lbm.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann library for
 * antiplane shear with dynamic mode III crack propagation
 * (Schlueter-Kuhn et al., "Dynamic Propagation of Mode III Cracks in a
 * Lattice Boltzmann Method for Solids", arXiv 2206.12412).
 *
 * One handle holds one lattice on one GPU.  Every time step is
 *   (1) the fused D2Q5 stream + collide + integrate update of all sites
 *       (Sec. 3: eqs. LBE, distrib-macro, f-eq, integration), with bounce-back
 *       on severed links and free edges and anti-bounce-back on Dirichlet
 *       edges (Sec. 3.1, link-local treatment of missing links);
 *   (2) optionally the macroscopic non-lattice-conforming rule on the crack
 *       boundary points (Sec. 3.1, eq. f-macro-bc);
 *   (3) the crack step of Alg. 1 (Sec. 4.1): K_III from the crack opening
 *       (Sec. 2.2, eq. sif; Sec. 4.2 evaluation window and eq. r(v)), the
 *       criterion (prescribed growth, or the K-criterion with the velocity of
 *       eq. v-tanh), tip advance by Delta a = adot dt, and severing of the
 *       links the new crack segment intersects.
 * All of it runs in this library's CUDA kernels, one kernel launch per time
 * step; the library owns the device state.  Conventions shared by every call:
 *   - every call returns lbm_status; nothing throws or exits across the ABI;
 *   - inputs are copied at create; no caller pointer is retained, except the
 *     allocator callbacks and their context, which must outlive the handle;
 *   - lbm_step only enqueues work on the handle's stream; calls that hand data
 *     to the host (lbm_fields to host memory, lbm_cut_mask, lbm_crack_state,
 *     lbm_sync) synchronise that stream.  The crack step that follows the last
 *     enqueued time step is applied (one small kernel) by the next call that
 *     reads or replaces the state, or by the next lbm_step;
 *   - a device-side error (a non-finite field) is sticky: every later call on
 *     the handle returns LBM_ERR_UNSTABLE;
 *   - lbm_last_error() describes the most recent failure on the calling thread;
 *   - a handle lives on the device that was current when it was created; make
 *     every call on it with that device current (the library does not switch
 *     devices).
 *
 * Geometry: sites sit at cell centres ((i + 1/2) dh, (j + 1/2) dh),
 * 0 <= i < nx, 0 <= j < ny; outer edges lie on half links.  Field planes are
 * exchanged as dense row-major ny x nx arrays (element (j, i) at j * nx + i).
 * The crack is a straight segment along +x on the line y = jc dh (jc an
 * integer), i.e. between rows jc-1 and jc; its tip is kept on a fixed-point
 * grid of 2^-32 dh.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument or unsupported configuration */
    LBM_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    LBM_ERR_OOM = -3,      /* the allocator returned NULL */
    LBM_ERR_UNSTABLE = -4, /* a non-finite value appeared in the fields or in K */
    LBM_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    LBM_ERR_STATE = -6,    /* call not valid in the handle's current state */
    LBM_ERR_IO = -7        /* file input/output failed */
} lbm_status;

/* edge kinds, one per outer edge */
enum { LBM_EDGE_FREE = 0, LBM_EDGE_DIRICHLET = 1, LBM_EDGE_PERIODIC = 2 };
/* edge indices into lbm_grid.edge and lbm_loading.edge */
enum { LBM_LEFT = 0, LBM_RIGHT = 1, LBM_BOTTOM = 2, LBM_TOP = 3 };
/* velocity sets.  LBM_D2Q5 (Sec. 3) is the method; LBM_D2Q9 (the paper notes
 * that the crack handling carries over to it, Sec. 4.1) adds the diagonal
 * links with equilibrium weights 2/3 g (axes) and 1/6 g (diagonals), the
 * isotropic nine-point Laplacian, stable for c_s^2 dt^2 / dh^2 <= 3/4.
 * D2Q9 is built with every bc_mode (with LBM_BC_MACROSCOPIC and
 * LBM_BC_MACROSCOPIC_EDGES a site that loses only a diagonal link to the
 * crack takes the normal of the crack face that link crosses, so every
 * crack-face point has the column-local rule of the crack faces; with
 * LBM_BC_MACROSCOPIC_EDGES the outer-edge points take the edge rule of the
 * D2Q5 lattice, along the edge's normal), FP64 or FP32 storage, in batches
 * of D2Q9 lattices and in row slabs (lbm_decomp.h: the crack rows inside one
 * slab), and not for lbm_tape_*.
 * Its diagonal links between rows jc-1 and jc cross the crack line at
 * x = (i + 1) dh and are severed when that point lies on the closed crack
 * segment; a diagonal link leaving the body through a corner follows the
 * Dirichlet edge if just one of the two is Dirichlet, else the bottom / top
 * edge. */
enum { LBM_D2Q5 = 0, LBM_D2Q9 = 1 };
enum { LBM_FORM_MOMENT = 0 };
/* storage of the fields.  LBM_F64: w and wdot in FP64, FP64 arithmetic.
 * LBM_F32: w and wdot in FP32, FP32 arithmetic.  LBM_F32_WD_BF16 /
 * LBM_F32_WD_F16: w in FP32, wdot stored in 16 bits (BF16, or FP16 holding
 * wdot * scale, see lbm_set_wd_scale), FP32 arithmetic; 12 bytes per site
 * update instead of 16.  LBM_F32_LEAPFROG: the state kept as w_n and w_{n-1}
 * in FP32 (the Euler integration of Sec. 3 makes wdot_n = (w_n - w_{n-1}) /
 * dt, eq. integration), FP32 arithmetic, w_{n+1} = w_n + ((w_n - w_{n-1}) +
 * g dt lap) written over w_{n-1}: 12 bytes per site update with FP32 state;
 * wdot is formed when read (LBM_FIELD_WDOT) and, when set, stored as
 * w_{n-1} = w_n - dt wdot against the current w (set W before WDOT).  D2Q5
 * with a crack along +x (not lbm_create_line, D2Q9 or tapes).  LBM_F64 and
 * LBM_F32 are also the dtype codes of field exchange. */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F32_WD_BF16 = 2, LBM_F32_WD_F16 = 3, LBM_F32_LEAPFROG = 4 };
/* treatment of the boundaries.  BOUNCEBACK: link-local rules on the crack
 * faces and the outer edges.  MACROSCOPIC: the macroscopic rule of Sec. 3.1
 * on the crack faces, link-local rules on the outer edges.
 * MACROSCOPIC_EDGES: the macroscopic rule on the crack faces and on every
 * free or Dirichlet outer edge (all boundaries, as in Sec. 5.2), see
 * lbm_lattice. */
enum { LBM_BC_BOUNCEBACK = 0, LBM_BC_MACROSCOPIC = 1, LBM_BC_MACROSCOPIC_EDGES = 2 };
/* crack modes (Alg. 1 "criterion") */
enum { LBM_CRACK_NONE = 0, LBM_CRACK_STATIONARY = 1, LBM_CRACK_PRESCRIBED = 2, LBM_CRACK_KCRIT = 3 };
/* loading kinds of a Dirichlet edge */
enum { LBM_LOAD_ZERO = 0, LBM_LOAD_LINEAR = 1, LBM_LOAD_SIN2 = 2, LBM_LOAD_HALFSINE = 3,
       LBM_LOAD_SERIES = 4, LBM_LOAD_CONST = 5 };
/* field planes */
enum { LBM_FIELD_W = 0, LBM_FIELD_WDOT = 1 };
/* cut masks */
enum { LBM_MASK_H = 0, LBM_MASK_V = 1 };
/* bits of lbm_crack_state_t.flags.  CLAMPED: the tip reached the body's
 * boundary and stopped.  UNSUPPORTED: with macroscopic faces on a crack in
 * any direction, a boundary point whose x_I or x_II cell reaches outside the
 * body came under the rule (its stencil is dropped, so its value is not the
 * rule's; the crack grew within two spacings of an edge).  NONFINITE: K or
 * the fields stopped being finite. */
enum { LBM_FLAG_CLAMPED = 1, LBM_FLAG_UNSUPPORTED = 2, LBM_FLAG_NONFINITE = 4 };

/* Lattice extent and spacing.  dh, dt > 0.  edge[] holds an LBM_EDGE_* per
 * edge index; periodic edges come in opposite pairs. */
typedef struct lbm_grid {
    int32_t nx, ny;
    double dh, dt;
    int32_t edge[4];
} lbm_grid;

/* Lattice model.  velocity_set = LBM_D2Q5 or LBM_D2Q9, form = LBM_FORM_MOMENT,
 * omega = dt / tau = 1 (the paper fixes tau = dt; Sec. 3).  storage is an
 * LBM_F64 / LBM_F32 / LBM_F32_WD_* code; bc_mode an LBM_BC_* code.
 *
 * LBM_BC_MACROSCOPIC_EDGES (Sec. 3.1, eq. f-macro-bc): after every LBM
 * update the boundary values w_B(t + dt) solve S w_B = R, each boundary
 * point's equation being a quadratic polynomial along the inward normal
 * evaluated at x_B.  An outer edge lies half a spacing outside its sites, so
 * x_B, x_I, x_II sit at 1/2, 3/2, 5/2 dh from it and x_I, x_II are the next
 * two sites: a traction-free edge gives w_B = (3 w_I - w_II) / 2, a
 * Dirichlet edge w_B = 8/15 w*(t + dt) + 2/3 w_I - 1/5 w_II.  A corner
 * between two such edges follows its Dirichlet edge, else the bottom / top
 * edge (the two choices differ only between two Dirichlet edges); a
 * site next to a severed crack link follows the crack face, whose x_I, x_II
 * on an edge column are edge points themselves.  wdot_B = (w_B(t + dt) -
 * w_B(t)) / dt.  One extra small kernel per time step applies it.  Needs at
 * least 4 sites across each non-periodic pair of edges and a crack line at
 * least 4 dh from the bottom and top edges (from a row slab's halo edge the
 * crack rows need only lie inside the slab).  Row slabs (lbm_decomp_*,
 * lbm_slab_*) apply it to each slab's own edge sites after the step, before
 * the boundary rows are exchanged; every slab then needs at least 4 rows.
 * Not available to lbm_tape_* (its create call rejects it). */
typedef struct lbm_lattice {
    int32_t velocity_set;
    int32_t form;
    double omega;
    int32_t storage;
    int32_t bc_mode;
} lbm_lattice;

/* Density and shear modulus; c_s = sqrt(mu / rho) (Sec. 2.1).  The update is
 * stable only for g = c_s^2 dt^2 / dh^2 <= 1/2 (D2Q5; 3/4 for D2Q9); larger g
 * is rejected. */
typedef struct lbm_material {
    double rho, mu;
} lbm_material;

/* Straight crack along +x on the line y (a multiple of dh, at least 3 dh from
 * the bottom and top edges, 4 dh with LBM_BC_MACROSCOPIC_EDGES), from
 * x_start to x_tip (physical units).
 * v_rel: prescribed relative speed adot / c_s (LBM_CRACK_PRESCRIBED).
 * K_C, v_max: K-criterion and eq. v-tanh (LBM_CRACK_KCRIT).
 * r0: eq. r(v); r_min > 0 overrides it with a fixed evaluation distance.
 * fit_width: width W of the evaluation window [r_min, r_min + W) (dh if <= 0).
 * hist_cap: capacity of the per-step history ring (records kept on device).
 * two_tips: 1 lets the end at x_start grow too, towards -x (a centre crack
 * with two tips, Sec. 5.2); each end runs the crack step of Alg. 1 with its
 * own speed memory, and the left end stops at x = 0.  0: only x_tip grows. */
typedef struct lbm_crack {
    int32_t mode;
    int32_t two_tips;
    double y, x_start, x_tip;
    double v_rel, K_C, v_max, r0, r_min, fit_width;
    int64_t hist_cap;
} lbm_crack;

/* Straight crack in any direction (Sec. 4.1: the crack is a line independent
 * of the lattice that grows along a given direction), from (x_start, y_start)
 * through the initial tip (x_tip, y_tip) (physical units, both in the closed
 * body [0, nx dh] x [0, ny dh], distinct), growing from the tip along the
 * unit direction c from the one to the other.  Both points are rounded to
 * the 2^-32 dh grid; every advance Delta a c is rounded to it per
 * component, and each step severs the H and V links that the segment from
 * the old to the new tip meets (closed segments, exact), so the crack is
 * the polyline of its tips; a tip that meets the body's boundary stops
 * there.  The crack's line must pass through no site centre.  K (eq. sif)
 * is fitted over the severed links whose midpoint m lies at
 * r = (x_tip - m) . c in [r_min, r_min + W), with the opening
 * w(left of c) - w(right of c) of the link's two sites; the window must
 * start more than dh / 2 behind the tip (r0 > dh / 2, or r_min > dh / 2).
 * two_tips: 1 lets the start grow too, along -c, with its own speed memory
 * and the same opening sign (a centre crack in that direction); its K window
 * lies along +c behind it.  The other fields are those of lbm_crack.  Built
 * for D2Q5 with every storage, LBM_BC_BOUNCEBACK (link-local faces) or
 * LBM_BC_MACROSCOPIC: the macroscopic rule (Sec. 3.1) on the crack's faces,
 * read for a crack off the lattice's axes -- a boundary point x_B takes the
 * normal n of the crack's line, x_I = x_B + n dh and x_II = x_B + 2 n dh are
 * interpolated bilinearly (their cells' corners all lie on x_B's side), and
 * the points coupled through those stencils are solved together to a
 * fixpoint.  LBM_ERR_ARG when a point of the initial crack has its x_I or
 * x_II cell outside the body; a point the crack reaches later with such a
 * cell drops that stencil (keep the crack two spacings from the edges).
 * The outer edges stay link-local. */
typedef struct lbm_crack_line {
    int32_t mode;
    int32_t two_tips;
    double x_start, y_start, x_tip, y_tip;
    double v_rel, K_C, v_max, r0, r_min, fit_width;
    int64_t hist_cap;
} lbm_crack_line;

/* Boundary value w*(t) of one Dirichlet edge:
 * LINEAR amp*min(t/t_ramp,1); SIN2 amp*sin^2(pi t/(2 t_ramp)) then amp
 * (Sec. 5.1); HALFSINE amp*sin(pi t/t_ramp) then 0 (Sec. 5.2); SERIES
 * series[n] at step n, holding the last value (copied at create); CONST amp.
 * The value at t_n = n dt is applied in the step t_n -> t_n+1. */
typedef struct lbm_loading {
    int32_t edge;
    int32_t kind;
    double amp;
    double t_ramp;
    const double *series;
    int64_t n_series;
} lbm_loading;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes aligned to 256 bytes,
 * or NULL; release frees it.  When NULL is passed, cudaMalloc / cudaFree are
 * used.  The library allocates device memory only inside lbm_create,
 * lbm_batch_create and lbm_tape_create (lbm_adjoint.h). */
typedef struct lbm_allocator {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*release)(void *ptr, void *ctx);
    void *ctx;
} lbm_allocator;

/* Crack state after the last completed step.  tip_q is the tip in units of
 * 2^-32 dh; n_cut counts severed crack links; r_min is the evaluation
 * distance used in the last K evaluation; npairs the number of site pairs
 * that entered it (0: K undefined, no growth). */
typedef struct lbm_crack_state_t {
    int64_t step, tip_q, n_cut, hist_n;
    double tip_x, K, v, r_min;
    int32_t npairs, flags;
} lbm_crack_state_t;

typedef struct lbm_handle lbm_handle;

/* Build a lattice on the current CUDA device.  stream (a cudaStream_t, NULL
 * for the legacy default stream) is where every later call enqueues work.
 * loads: n_loads entries, at most one per edge; a Dirichlet edge without an
 * entry is held at w* = 0.  The fields start at w = wdot = 0 with the initial
 * crack's links severed.  Returns LBM_ERR_ARG for invalid input (non-positive
 * sizes, g > 1/2, omega != 1, a crack outside the lattice, unpaired periodic
 * edges, periodic left/right edges with macroscopic crack faces). */
lbm_status lbm_create(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                      const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads,
                      void *stream, const lbm_allocator *allocator, lbm_handle **out);

/* The same with a straight crack in any direction (lbm_crack_line; crack
 * must not be NULL and its mode not LBM_CRACK_NONE).  Every call below
 * applies to the handle (lbm_set_launch sets the march bands of its step;
 * lbm_batch_create takes it in a batch of such lattices), except the row
 * slabs (lbm_decomp.h) and the adjoint (lbm_adjoint.h), which return
 * LBM_ERR_ARG or LBM_ERR_STATE.  In
 * lbm_crack_state (lbm_crack_state_left: the start of a two-tip crack),
 * tip_q and tip_x are the end's x and n_cut counts the severed links;
 * lbm_line_tip (lbm_line_tip_left) gives its y.
 * LBM_ERR_ARG for the cases listed at lbm_crack_line. */
lbm_status lbm_create_line(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                           const lbm_crack_line *crack, const lbm_loading *loads, int32_t n_loads,
                           void *stream, const lbm_allocator *allocator, lbm_handle **out);

/* The tip of a crack in any direction: x and y in units of 2^-32 dh (either
 * pointer may be NULL) and, if y_hist is not NULL, the y of the last
 * min(cap, hist_n, hist_cap) per-step records in chronological order (their
 * x, K, v and pairs come from lbm_crack_state); *n_written receives the
 * number of records.  LBM_ERR_STATE for a handle without such a crack.
 * Synchronises the stream. */
lbm_status lbm_line_tip(lbm_handle *h, int64_t *x_q, int64_t *y_q, int64_t *y_hist, int64_t cap, int64_t *n_written);

/* The same for the start of a two-tip crack in any direction (its growing
 * left end); LBM_ERR_STATE if the crack has one growing end. */
lbm_status lbm_line_tip_left(lbm_handle *h, int64_t *x_q, int64_t *y_q, int64_t *y_hist, int64_t cap,
                             int64_t *n_written);

/* Enqueue n >= 0 time steps (each: bulk update, crack-face rule, crack step)
 * on the handle's stream.  Asynchronous; errors of the device work surface at
 * the next synchronising call. */
lbm_status lbm_step(lbm_handle *h, int64_t n);

/* Copy field `which` (LBM_FIELD_W or LBM_FIELD_WDOT) as a dense ny x nx
 * row-major array into dst, which lies in device memory if dst_on_device,
 * else in host memory (then the stream is synchronised before returning).
 * dtype is LBM_F64 for F64 storage and LBM_F32 for every other storage
 * (16-bit wdot planes are converted to FP32). */
lbm_status lbm_fields(lbm_handle *h, int32_t which, void *dst, int32_t dst_on_device, int32_t dtype);

/* Overwrite field `which` from a dense ny x nx row-major array of dtype
 * (as for lbm_fields; FP32 input is rounded to a 16-bit wdot plane).  Crack,
 * step counter and history are left unchanged. */
lbm_status lbm_set_fields(lbm_handle *h, int32_t which, const void *src, int32_t src_on_device, int32_t dtype);

/* lbm_fields / lbm_set_fields for an ny x nx array whose rows lie row_stride
 * >= nx elements apart (for example nx columns of a wider array): element
 * (j, i) at dst[j * row_stride + i].  The same fields (w, wdot of Sec. 3:
 * the state (w, wdot) that the moment form of the update advances), the
 * same dtype rule, the same host/device and synchronisation rules; the
 * elements between rows are left untouched.  row_stride == nx is the dense
 * call; row_stride < nx returns LBM_ERR_ARG. */
lbm_status lbm_fields_strided(lbm_handle *h, int32_t which, void *dst, int32_t dst_on_device, int32_t dtype,
                              int64_t row_stride);
lbm_status lbm_set_fields_strided(lbm_handle *h, int32_t which, const void *src, int32_t src_on_device, int32_t dtype,
                                  int64_t row_stride);

/* Copy a cut mask into host memory: row j occupies words_per_row =
 * ceil(nx / 32) words starting at j * words_per_row; bit b of word w is
 * column 32 w + b.  LBM_MASK_H bit (i, j): link (i,j)-(i+1,j) severed (i =
 * nx-1: the periodic wrap link); LBM_MASK_V bit (i, j): link (i,j)-(i,j+1).
 * n_words must be at least ny * words_per_row.  Synchronises the stream. */
lbm_status lbm_cut_mask(lbm_handle *h, int32_t which, uint32_t *dst_host, int64_t n_words);

/* Current crack state, plus (if the pointers are not NULL) the last
 * min(cap, hist_n, hist_cap) per-step records in chronological order: K,
 * relative speed v, tip_q and number of pairs.  *n_written receives the
 * number of records copied.  Synchronises the stream. */
lbm_status lbm_crack_state(lbm_handle *h, lbm_crack_state_t *now, double *K_hist, double *v_hist,
                           int64_t *tip_hist, int32_t *npairs_hist, int64_t cap, int64_t *n_written);

/* The same for the left end of a two-tip crack (tip_q, tip_x, K, v, r_min,
 * npairs, flags of that end; step, n_cut and hist_n are shared).
 * LBM_ERR_STATE if the crack has one growing end. */
lbm_status lbm_crack_state_left(lbm_handle *h, lbm_crack_state_t *now, double *K_hist, double *v_hist,
                                int64_t *tip_hist, int32_t *npairs_hist, int64_t cap, int64_t *n_written);

/* Synchronise the handle's stream and report sticky device errors. */
lbm_status lbm_sync(lbm_handle *h);

/* Move later work to another stream (the caller orders the two streams). */
lbm_status lbm_set_stream(lbm_handle *h, void *stream);

/* Launch shape of the step kernel (D2Q5, D2Q9 and a crack in any
 * direction).  Each CTA marches over a band of at most band_rows rows of one
 * column block; 0 picks the built-in partition (D2Q5 and a crack in any
 * direction: the shortest bands for which every CTA of a step is resident at
 * once; D2Q9: about three waves of shorter bands).  The rows
 * next to the crack line (jc-3 .. jc+2 with macroscopic crack faces, jc-1 and
 * jc otherwise) always form two bands of their own.  Synchronises the stream
 * and drops the cached step graph. */
lbm_status lbm_set_launch(lbm_handle *h, int32_t band_rows);

/* Current launch shape: the longest band, the number of CTAs, threads per CTA
 * and how many CTAs of the step kernel an SM holds (any pointer may be NULL). */
lbm_status lbm_get_launch(const lbm_handle *h, int32_t *band_rows, int32_t *ctas, int32_t *threads,
                          int32_t *ctas_per_sm);

/* The solve of the macroscopic rule on the faces of a crack in any direction
 * (lbm_create_line with LBM_BC_MACROSCOPIC; Sec. 3.1, S w_B = R).  mode 0
 * (default): the chunked solve -- one CTA per 256 consecutive boundary
 * entries along the line, each solving its entries and the entries they
 * depend on level by level (a point's stencil corners lie strictly farther
 * from the line, so the coupling is acyclic apart from the point's own site)
 * -- wherever the coupling is at most 64 levels deep, else the one-CTA
 * solve; mode 1: always the one-CTA Jacobi solve to a bitwise fixpoint.
 * Both give the rule's solution (not the same last bits).  *chunked (may be
 * NULL) tells which one runs.  Synchronises the stream; no effect on other
 * lattices. */
lbm_status lbm_set_face_solve(lbm_handle *h, int32_t mode, int32_t *chunked);

/* How the step kernel's interior CTAs (no edge row or column, not the crack
 * rows) read their rows.  enable = 0 (default): each thread loads its row
 * segments into registers one row ahead.  enable = 1: the CTA stages them in
 * a ring of shared-memory slots filled by bulk asynchronous copies
 * (cp.async.bulk on mbarriers) up to four rows ahead, so the bytes in flight
 * do not depend on the number of resident warps.  The arithmetic is the same
 * (identical results).  Taken only for FP32 w storage (LBM_F32 and the
 * 16-bit wdot forms), D2Q5 and a crack along +x; ignored otherwise.  Every
 * wait of the staged path is bounded: a copy that does not arrive within a
 * clock budget (about a second) ends the launch with LBM_ERR_TIMEOUT at the
 * next synchronising call.  Synchronises the stream and re-partitions the
 * rows for the chosen kernel's occupancy (as lbm_set_launch(h, 0)). */
lbm_status lbm_set_bulk(lbm_handle *h, int32_t enable);

/* How consecutive kernels of the time steps are launched.  enable != 0:
 * chained by programmatic dependent launch -- the CTAs of a step's kernel
 * (and of the edge-rule, face and crack-face kernels that follow it) are
 * dispatched while the kernel before it still runs and wait on the device
 * for it to complete, so no launch gap separates the steps of a lattice.
 * enable = 0: plain launches.  The default is chained for lattices of at most
 * 2^18 sites, whose steps take a few microseconds and are bound by launch
 * latency, and plain for larger ones, where early-resident CTAs of the next
 * step cost more than the gap they save.  The arithmetic is the same
 * (identical results).  Synchronises the stream and drops the cached step
 * graph.  lbm_batch_set_chained does the same for a batch's launches (plain
 * by default).  No counterpart in the paper. */
lbm_status lbm_set_chained(lbm_handle *h, int32_t enable);

/* Kernel timing: while enabled, lbm_step launches every step directly (no
 * graph) with CUDA events on the handle's stream around the step kernel, and
 * the deferred crack step that synchronising calls apply first is timed the
 * same way. */
lbm_status lbm_set_profiling(lbm_handle *h, int32_t enable);

/* Sum of the measured kernel durations (milliseconds) and launch counts since
 * the last reset, for step kernels and for deferred crack steps; reset != 0
 * clears them.  Synchronises the stream. */
lbm_status lbm_profile_read(lbm_handle *h, double *step_ms, int64_t *n_step, double *finalize_ms, int64_t *n_finalize,
                            int32_t reset);

/* Return to the state lbm_create left: w = wdot = 0, step 0, the initial
 * crack (mask, tip and crack state), an empty history.  The current loads,
 * launch shape and FP16 scale are kept; a sticky error is not cleared.
 * Synchronises the stream. */
lbm_status lbm_reset(lbm_handle *h);

/* Replace the loading of one edge (load->edge) from the next step on; the
 * value w*(t_n) of the current step n is recomputed.  A SERIES load may be at
 * most as long as the series that edge was created with (its device buffer is
 * reused; an edge created without a series cannot take one).  The FP16
 * scale is not re-derived.  Not for a lattice held by a batch.  Synchronises
 * the stream and drops the cached step graph. */
lbm_status lbm_set_loading(lbm_handle *h, const lbm_loading *load);

/* Scale of FP16 wdot storage (LBM_F32_WD_F16): the plane holds wdot * scale.
 * scale must be a power of two; the stored plane is rescaled.  lbm_create
 * picks 2^(10 - ceil(log2 r)), r the largest rate of change of the edge values
 * (1024 without loads), so that waves up to 64 times that rate fit.  A value
 * that overflows FP16 becomes infinite and is reported as LBM_ERR_UNSTABLE.
 * Returns LBM_ERR_STATE for other storages. */
lbm_status lbm_set_wd_scale(lbm_handle *h, double scale);
lbm_status lbm_get_wd_scale(const lbm_handle *h, double *scale);

/* Copy the wdot plane of a lattice with 16-bit wdot storage
 * (LBM_F32_WD_BF16 / LBM_F32_WD_F16) into host memory as a dense ny x nx FP32
 * array -- the same values lbm_fields(h, LBM_FIELD_WDOT, dst, 0, LBM_F32)
 * gives -- without allocating and without the handle's staging buffer: the
 * conversion runs into one fixed device array of 2^20 floats (4 MiB) that
 * belongs to the library.  The paper has no counterpart (this is a
 * memory-management variant of a copy-out).  It is meant for callers that
 * cannot allocate device memory at the point where they read the field: an
 * application whose device memory is fully committed to its own pools (an
 * allocation would fail, or would first make the caching allocator release
 * and synchronise), or code that reads the field between steps inside a loop
 * that must not call into an allocator at all.  Limits and rules:
 *   - lattices of at most 2^20 sites (LBM_ERR_ARG beyond); n_floats >= nx*ny;
 *   - LBM_ERR_STATE for other storages (use lbm_fields);
 *   - like every call on a handle, it is not safe to make it while another
 *     thread makes a call on the same handle (it applies the pending crack
 *     step, changes the handle's bookkeeping and enqueues work on its
 *     stream): serialise it with the handle's other calls, e.g. make it from
 *     the thread that steps the lattice, between its lbm_step calls;
 *   - the array's address is looked up on each call made outside a stream
 *     capture; during a capture the last lookup on the device is used, so the
 *     first call on a device must come before any stream capture;
 *   - the array is shared by every call on the device, whichever handle:
 *     calls that overlap on the GPU (from several threads, or on several
 *     streams) race on it and must be serialised by the callers;
 *   - nothing in the array needs to start at zero (a call reads back only
 *     what it wrote);
 *   - synchronises the handle's stream; applies the pending crack step first,
 *     as lbm_fields does. */
lbm_status lbm_wdot_to_host_noalloc(lbm_handle *h, float *dst_host, int64_t n_floats);

/* Checkpoint / resume.  lbm_save writes the whole state of the lattice to
 * the file `path`: w and the stored wdot (padded planes, bit for bit), the
 * cut masks, the crack state (both ends, after the pending crack step is
 * applied), the history ring, the step counter (the loads' time) and the
 * FP16 wdot scale, behind a header that records the configuration.  lbm_load
 * reads such a file into a handle created with the same grid, lattice,
 * material, crack and loads (LBM_ERR_ARG otherwise); stepping on from there
 * gives the same bits as the run that was saved.  The paper has no
 * counterpart (its runs are single programs).  Both synchronise the stream;
 * LBM_ERR_IO when the file cannot be written or read, or is truncated or
 * not a checkpoint. */
lbm_status lbm_save(lbm_handle *h, const char *path);
lbm_status lbm_load(lbm_handle *h, const char *path);

/* Bytes of device memory the handle holds. */
lbm_status lbm_device_bytes(const lbm_handle *h, int64_t *bytes);

/* Release the handle and its device memory (NULL is ignored).  Synchronises
 * the stream first.  Destroy any batch that holds the handle first. */
void lbm_destroy(lbm_handle *h);

/* ---- Batches: many independent lattices advanced by one kernel launch per
 * time step (each lattice's time step exactly as lbm_step computes it, so a
 * batched lattice ends bit-identical to the same lattice stepped alone).
 *
 * lbm_batch_create groups n existing handles (not owned; they must outlive
 * the batch) of the same storage, on the same stream, stepped equally often.
 * It re-partitions every lattice into bands of band_rows rows (0: 16; -1:
 * the balanced step of lbm_batch_set_shape) and
 * uploads a table of the step-kernel arguments of every lattice and a table
 * of all their (lattice, column block, band) units; allocator as in
 * lbm_create (NULL: cudaMalloc).  All lattices of one velocity set: D2Q5,
 * or D2Q9 (a D2Q9 batch takes CTAs of 128 threads over bands, a lookahead of
 * one row, no balanced and no persistent form; its lattices with the
 * macroscopic rule on their crack faces get it from one more batched launch
 * per step, units of 128 columns); or lattices with a crack in any direction
 * (lbm_create_line; all members of that kind: each keeps its own fixed
 * line-step grid, the batch takes CTAs of 128 threads and a lookahead of one
 * row, band_rows is ignored, there is no balanced and no persistent form, and
 * each lattice with the macroscopic rule on its faces runs its face solve as
 * its own launch after the batched step).  Lattices with
 * LBM_BC_MACROSCOPIC_EDGES get their outer-edge rule from one more batched
 * launch per step (units of 128 edge sites).  While the batch exists, step its lattices
 * only through lbm_batch_step (stepping one alone makes lbm_batch_step return
 * LBM_ERR_STATE) and do not call lbm_set_launch or lbm_set_wd_scale on them.
 * Fields, masks and crack states are read through the member handles. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(lbm_handle *const *handles, int32_t n, int32_t band_rows, const lbm_allocator *allocator,
                            lbm_batch **out);

/* Create n lattices (member i as lbm_create(&grids[i], &lattices[i],
 * &materials[i], cracks ? &cracks[i] : NULL, loads ? loads[i] : NULL,
 * n_loads ? n_loads[i] : 0, stream, allocator)) and group them as
 * lbm_batch_create(..., band_rows, allocator) does.  The batch owns them:
 * lbm_batch_destroy destroys them too (lbm_batch_member gives each handle,
 * for reading fields, masks and crack states; do not destroy those handles).
 * The paper has no batches: many independent runs of the method (Sec. 3,
 * Alg. 1), each exactly as one lattice, advance in one launch per step.
 * loads and n_loads are both NULL or both given.  On error nothing is left
 * allocated and the message names the member that failed. */
lbm_status lbm_create_batch(int32_t n, const lbm_grid *grids, const lbm_lattice *lattices, const lbm_material *materials,
                            const lbm_crack *cracks, const lbm_loading *const *loads, const int32_t *n_loads,
                            void *stream, const lbm_allocator *allocator, int32_t band_rows, lbm_batch **out);

/* Member i (0 <= i < n) of a batch: the handle, in the order given at
 * create.  LBM_ERR_ARG for an index out of range. */
lbm_status lbm_batch_member(const lbm_batch *b, int32_t i, lbm_handle **h);

/* Enqueue n >= 0 time steps of every lattice of the batch on the shared
 * stream (CUDA-graph replay of 64-step chunks). */
lbm_status lbm_batch_step(lbm_batch *b, int64_t n);

/* Number of lattices and CTAs per step of the batch (pointers may be NULL). */
lbm_status lbm_batch_info(const lbm_batch *b, int32_t *n_lattices, int32_t *ctas);

/* Launch shape of the batched step: CTAs of `threads` threads (32, 64 or 128;
 * a column block is threads 16-byte vectors wide, i.e. 4 * threads FP32
 * columns) over bands of band_rows >= 1 rows (the crack rows keep bands of
 * their own), or with band_rows = 0 bands as tall as one wave of resident
 * CTAs allows, about equally tall in every lattice (long marches, few halo
 * rows, no second wave), or with band_rows = -1 the balanced step: as many
 * CTAs as are resident at once, each marching a run of row pieces of about
 * the same total height (a lattice's rows outside its crack sub-bands are cut
 * into row blocks of about one CTA's share, column block by column block, and
 * that sequence into one run per CTA; the crack sub-bands stay units of their
 * own), so that lattices of any heights fill one wave evenly; lbm_batch_info
 * then reports those CTAs; or with band_rows = -2 tapered bands: the
 * lattices' units are launched largest lattice first, in bands of 48 rows,
 * and the smallest lattices holding the last sixth of the sites take bands
 * of 8 rows, so that the units handed out last are short.  Narrow column blocks leave fewer idle warps right of lattices
 * whose width is not a multiple of 512 columns; short bands give more CTAs.
 * The results do not depend on the shape (each lattice's time step is the
 * same arithmetic).  lbm_batch_set_shape synchronises the stream and
 * re-partitions every member lattice; lbm_batch_get_shape reads it back.
 * The paper has no counterpart (its runs are single lattices). */
lbm_status lbm_batch_set_shape(lbm_batch *b, int32_t threads, int32_t band_rows);
lbm_status lbm_batch_get_shape(const lbm_batch *b, int32_t *threads, int32_t *band_rows);

/* Row lookahead of the batched step's march: with rows = 1 (the default) a
 * warp keeps the loads of the row after next in flight while it updates a
 * row; with rows = 2 it keeps two rows of loads in flight (eight more
 * registers a thread, so 28 instead of 32 resident warps per SM), which
 * hides more of the memory latency of short bands.  Same arithmetic: the
 * results do not depend on it.  rows other than 1 or 2: LBM_ERR_ARG.
 * lbm_batch_set_lookahead synchronises the stream and re-partitions (the
 * single-wave band heights of band_rows = 0 depend on the resident CTAs);
 * lbm_batch_get_lookahead reads it back.  No counterpart in the paper. */
lbm_status lbm_batch_set_lookahead(lbm_batch *b, int32_t rows);
/* Chained launches of the batched step (as lbm_set_chained; default off). */
lbm_status lbm_batch_set_chained(lbm_batch *b, int32_t enable);
lbm_status lbm_batch_get_lookahead(const lbm_batch *b, int32_t *rows);

/* Autotuner of the batched step's launch shape: times trial_steps (2..1024)
 * batched steps with CUDA events for every shape of lookahead in {1, 2} x
 * threads in {32, 64, 128} x band_rows in {-1 (balanced), 0 (one wave), 8, 16,
 * 32, 64, -2 (tapered)}
 * (the first of three repetitions a warm-up), keeps the fastest (its
 * lookahead is read back with lbm_batch_get_lookahead), and caches it in the process under the device's SM
 * count, the storage and the lattices' sizes and crack rows (a later batch of
 * the same lattices takes the cached shape without trials; *from_cache = 1,
 * *us_per_step = 0).  The trials advance the lattices, so the tuner first
 * applies any pending crack step, copies every member's device state to a
 * scratch allocation of the same total size (from the batch's allocator;
 * LBM_ERR_OOM if it fails) and copies it back afterwards: the lattices end as
 * they were.  Synchronises the stream.  Outputs may be NULL. */
lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, int32_t *threads, int32_t *band_rows,
                          double *us_per_step, int32_t *from_cache);

/* Persistent form of the batched step.  With enable != 0, lbm_batch_step(b,
 * n) enqueues ONE cooperative launch (CTAs of the batch's shape, as many as
 * are resident at once) that runs all n steps: each CTA takes every
 * grid-size-th unit of a step, then every CTA meets at a grid barrier before
 * the next step (and before the edge-rule units of a step).  A CTA waits at
 * most budget_cycles clock cycles (0: 2^31, about 1 s) at a barrier; then
 * it sets a timeout flag in every member lattice and returns, and the
 * others give up at their next wait, so the launch always ends.  The next
 * call that synchronises a member handle then returns LBM_ERR_TIMEOUT (and
 * the handle stays in that error state).  Results are bit-identical to the
 * per-step launches (enable = 0, the default: graph replay of one launch per
 * step).  No counterpart in the paper. */
lbm_status lbm_batch_set_persistent(lbm_batch *b, int32_t enable, int64_t budget_cycles);

/* Diagnostic of the bounded device wait used by the persistent batched
 * step: `ctas` CTAs (1..64) of a small kernel on `stream` meet at a grid
 * barrier that expects `expected` (1..64) arrivals, each waiting at most
 * budget_cycles (1e3..2^34) clock cycles.  Returns LBM_OK if the barrier
 * completed for every CTA and LBM_ERR_TIMEOUT if a wait gave up (as it must
 * when ctas < expected: nothing completes the barrier).  Allocates 256 bytes
 * of device memory for the call; synchronises the stream. */
lbm_status lbm_barrier_probe(int32_t ctas, int32_t expected, int64_t budget_cycles, void *stream);

/* Release the batch (NULL is ignored); the member handles stay valid. */
void lbm_batch_destroy(lbm_batch *b);

/* Message of the most recent failure on the calling thread ("" if none).
 * The pointer stays valid until the next call on this thread. */
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
