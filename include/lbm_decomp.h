/*
 * lbm_decomp.h -- a lattice split into row slabs ("virtual ranks") on one
 * GPU, each slab its own lattice, with the halo rows exchanged after every
 * step.
 *
 * The time step of Sec. 3 reads, at each site, only the four neighbours' w
 * (the moment form), so a lattice split into slabs of whole rows needs, per
 * step and per inner boundary, one row of w from each side: each slab keeps
 * its neighbour's boundary row in its pad row beyond the boundary (its halo
 * row).  The crack's rows (the sub-bands jc-3 .. jc-1 and jc .. jc+2 with the
 * macroscopic crack-face rule of Sec. 3.1, jc-1 and jc with bounce-back) lie
 * inside one slab, or the crack line itself is the boundary between two
 * slabs, each holding its side's sub-band.  In the second case both slabs
 * run the crack step of Alg. 1: the site pairs of the K_III fit (eq. sif;
 * rows jc-1 and jc) are one own row and the halo row on either side, so both
 * form the same sums in the same order, reach the same K, the same decision
 * and the same severed links (each slab keeps its copy of the crack state
 * and of the crack row of the cut mask).  With LBM_BC_MACROSCOPIC_EDGES each
 * slab applies the edge rule to its own edge sites (the left and right edge
 * points of its rows; the bottom / top edge and corners in the first / last
 * slab; the crack-face points on the edge columns, whose x_I, x_II are edge
 * points of the same slab) after its step and before the exchange: every
 * equation reads sites of its own row, or of rows of the same slab, and
 * slabs take at least 4 rows.  A D2Q9 lattice (LBM_D2Q9) splits the same
 * way: its nine-point update reads rows j-1, j, j+1 only, so the one halo
 * row per side still carries everything (the diagonal neighbours are sites
 * of that row); its crack rows stay inside one slab (its diagonal cuts, its
 * crack step and its crack-face rule read both sides of the crack line), so
 * no boundary may lie on the crack line.  No other data crosses a boundary:
 * a decomposed run is bit-identical to the undivided one.  The paper runs on
 * one process.  lbm_decomp_* keeps all slabs on one device (one batched
 * launch and one row-exchange launch per step); lbm_slab_* gives one slab to
 * each process (or device), which exchange the boundary rows themselves.
 * Conventions are those of lbm.h.
 */
#ifndef LBM_DECOMP_H
#define LBM_DECOMP_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_decomp lbm_decomp;

/* Row starts of a split of ny rows into n_ranks slabs: near-even slabs of at
 * least 2 rows whose boundaries avoid the crack rows [jc - hh, jc + hh)
 * except the crack line jc itself (a boundary that falls strictly inside
 * moves to the nearest of jc - hh, jc and jc + hh); jc < 0 means no crack.  hh = 3 with macroscopic crack faces, 1 with bounce-back.
 * This is the D2Q5 split; lbm_decomp_create plans a D2Q9 lattice's split
 * itself, moving a boundary to the nearer of jc - hh and jc + hh.
 * Writes n_ranks + 1 values (0 first, ny last) to row_start (host memory).
 * LBM_ERR_ARG if no such split exists.  Host-only; touches no device. */
lbm_status lbm_decomp_plan(int32_t ny, int32_t jc, int32_t hh, int32_t n_ranks, int32_t *row_start);

/* Build the lattice of lbm_create as n_ranks slabs (arguments as for
 * lbm_create; storage any the lattice takes).  row_start: n_ranks + 1
 * ascending row indices from 0 to ny with every slab at least 2 rows and no
 * boundary inside the crack rows but, for D2Q5, the crack line (then with
 * the hh rows of each side in its slab), or NULL for the planned split.  Slab r holds rows row_start[r]
 * .. row_start[r+1]-1; its inner bottom/top edges are halo edges, its other
 * edges and loads those of the lattice; with FP16 wdot storage every slab
 * takes the scale the undivided lattice would.  LBM_ERR_ARG for bad input. */
lbm_status lbm_decomp_create(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                             const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads, int32_t n_ranks,
                             const int32_t *row_start, void *stream, const lbm_allocator *allocator,
                             lbm_decomp **out);

/* Enqueue n >= 0 time steps of every slab plus the halo exchange after each
 * (CUDA-graph replay of 64-step chunks). */
lbm_status lbm_decomp_step(lbm_decomp *d, int64_t n);

/* Field `which` of the whole lattice as a dense ny x nx array (gathered from
 * the slabs), as lbm_fields. */
lbm_status lbm_decomp_fields(lbm_decomp *d, int32_t which, void *dst, int32_t dst_on_device, int32_t dtype);

/* Overwrite field `which` of the whole lattice from a dense ny x nx array
 * (scattered to the slabs, halo rows refreshed), as lbm_set_fields. */
lbm_status lbm_decomp_set_fields(lbm_decomp *d, int32_t which, const void *src, int32_t src_on_device, int32_t dtype);

/* Slab r: its handle (owned by the decomposition: read it -- fields, crack
 * state, masks -- but do not step it, re-launch it or destroy it), its first
 * row and its row count (any pointer may be NULL).  crack_rank receives the
 * slab that holds the crack (-1 without a crack). */
lbm_status lbm_decomp_rank(const lbm_decomp *d, int32_t rank, lbm_handle **slab, int32_t *row0, int32_t *rows);
lbm_status lbm_decomp_info(const lbm_decomp *d, int32_t *n_ranks, int32_t *crack_rank);

/* Release the slabs and the decomposition (NULL is ignored). */
void lbm_decomp_destroy(lbm_decomp *d);

/* ---- One slab per process.  lbm_slab_create builds rows row0 .. row0+rows-1
 * of the lattice lbm_create would build (same arguments, plus the slab's
 * rows; rows >= 2) as a lattice of its own on `stream`: its bottom (top)
 * edge is a halo edge when row0 > 0 (row0 + rows < ny) or the lattice is
 * periodic in y, otherwise the lattice's edge with its load.  The crack goes
 * to the slab when the crack line lies inside it or on one of its halo
 * boundaries (LBM_ERR_ARG when a boundary cuts the crack rows elsewhere, or
 * the slab lacks its side's crack rows; for D2Q9, when a boundary cuts the
 * crack rows at all, the crack line included).  FP16 wdot storage takes the scale
 * of the undivided lattice.  The handle is an ordinary lattice handle (step,
 * read, checkpoint and destroy it with the lbm.h calls; no batches or
 * tapes).
 *
 * Every step of a slab reads its halo rows: the neighbours' boundary rows of
 * the state it advances.  So after set_fields and after every lbm_step(h, 1),
 * and before any other call on the handle, the caller exports the slab's
 * boundary rows (lbm_slab_export), delivers each to the neighbour across
 * that boundary (any transport), and imports the neighbours' rows
 * (lbm_slab_import).  Both calls copy nx values of w in the storage's
 * arithmetic type (FP64 for LBM_F64, else FP32), dense, and neither applies
 * the pending crack step (that step reads the halo row, which must be in
 * place first).  side 0: the bottom row (export) / the halo below row 0
 * (import); side 1: the top row / the halo above it.  Host buffers make the
 * call synchronise the stream; device buffers are stream-ordered on the
 * slab's stream.  lbm_slab_import returns LBM_ERR_ARG for a side that is an
 * outer edge.  Stepped this way, every slab is bit-identical to its rows of
 * the undivided lattice, and slabs on both sides of the crack line report
 * the same crack state and history. */
lbm_status lbm_slab_create(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                           const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads, int32_t row0,
                           int32_t rows, void *stream, const lbm_allocator *allocator, lbm_handle **out);
lbm_status lbm_slab_export(lbm_handle *h, int32_t side, void *dst, int32_t dst_on_device);
lbm_status lbm_slab_import(lbm_handle *h, int32_t side, const void *src, int32_t src_on_device);

#ifdef __cplusplus
}
#endif

#endif /* LBM_DECOMP_H */
