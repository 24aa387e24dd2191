// lbm_decomp.cu -- host runtime behind include/lbm_decomp.h: the row-slab
// split, the slab lattices (halo edges inside), one batched step launch for
// all slabs and one row-exchange launch per step, replayed as CUDA graphs.
#include "lbm_decomp.h"
#include "lbm_host.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace lbm;
using namespace lbm::host;

struct lbm_decomp {
    std::vector<lbm_handle *> slabs;
    std::vector<int32_t> row_start;
    int crack_rank;
    lbm_batch *batch;
    int32_t nx, ny;
    size_t esize;
    int64_t row_bytes;      // one padded row of w
    RowCopy *pairs;         // device: [2 parities][n_pairs]
    int n_pairs;
    lbm_allocator alloc;
    bool custom_alloc;
    cudaStream_t stream, cap;
    ChunkGraph graph;
};

namespace {

// An inner boundary may not cut the crack's rows [jc - hh, jc + hh) except
// on the crack line itself (line_ok: D2Q5), where the slabs on both sides
// each hold their side's hh rows.  A D2Q9 lattice keeps all 2 hh rows in one
// slab: its diagonal cuts, crack step and face rule read both sides.
bool boundary_ok(int32_t b, int32_t below, int32_t above, int32_t jc, int32_t hh, bool line_ok = true)
{
    if (jc < 0 || b <= jc - hh || b >= jc + hh) return true;
    return line_ok && b == jc && below >= hh && above >= hh;
}

bool valid_split(int32_t ny, int32_t jc, int32_t hh, int32_t n, const int32_t *rs, bool line_ok = true)
{
    if (rs[0] != 0 || rs[n] != ny) return false;
    for (int r = 0; r < n; ++r)
        if (rs[r + 1] - rs[r] < 2) return false;
    for (int r = 1; r < n; ++r)
        if (!boundary_ok(rs[r], rs[r] - rs[r - 1], rs[r + 1] - rs[r], jc, hh, line_ok)) return false;
    return true;
}

// Even slabs, each inner boundary that would cut the crack rows moved to the
// nearest allowed row (an end of the crack rows, or the crack line itself
// when line_ok).
lbm_status plan_split(int32_t ny, int32_t jc, int32_t hh, int32_t n_ranks, int32_t *row_start, bool line_ok)
{
    if (!row_start) return fail(LBM_ERR_ARG, "row_start is NULL");
    if (n_ranks < 1 || ny < 2 * n_ranks) return fail(LBM_ERR_ARG, "need 1 <= n_ranks <= ny / 2");
    if (jc >= 0 && (hh < 0 || jc - hh < 0 || jc + hh > ny)) return fail(LBM_ERR_ARG, "crack rows outside the lattice");
    std::vector<int32_t> rs((size_t)n_ranks + 1);
    for (int r = 0; r <= n_ranks; ++r) {
        int32_t b = (int32_t)(((int64_t)r * ny + n_ranks / 2) / n_ranks);
        if (jc >= 0 && r > 0 && r < n_ranks && b > jc - hh && b < jc + hh && !(line_ok && b == jc)) {
            // the nearest of the crack rows' ends (and the crack line itself)
            const int32_t c[3] = {jc - hh, line_ok ? jc : jc + hh, jc + hh};
            int32_t best = c[0];
            for (int q = 1; q < 3; ++q)
                if (std::abs(c[q] - b) < std::abs(best - b)) best = c[q];
            b = best;
        }
        rs[(size_t)r] = b;
    }
    if (!valid_split(ny, jc, hh, n_ranks, rs.data(), line_ok))
        return fail(LBM_ERR_ARG, line_ok ? "no split into slabs of >= 2 rows keeps each side's crack rows in one slab"
                                         : "no split into slabs of >= 2 rows keeps the crack rows in one slab");
    std::copy(rs.begin(), rs.end(), row_start);
    clear_error();
    return LBM_OK;
}

// First byte of padded row j of buffer p of slab h.
char *row_ptr(const lbm_handle *h, int p, int j, size_t esize)
{
    const int64_t xoff = 128 / (int64_t)esize;
    return static_cast<char *>(h->w[p]) + ((int64_t)j * h->pitch - xoff) * (int64_t)esize;
}

void free_decomp(lbm_decomp *d)
{
    d->graph.reset();
    if (d->batch) lbm_batch_destroy(d->batch);
    for (lbm_handle *h : d->slabs) lbm_destroy(h);
    if (d->pairs) {
        if (d->custom_alloc) d->alloc.release(d->pairs, d->alloc.ctx);
        else cudaFree(d->pairs);
    }
    if (d->cap) cudaStreamDestroy(d->cap);
    delete d;
}

// Fill the halo rows of buffer p from the neighbours' boundary rows.
cudaError_t exchange(const lbm_decomp *d, int p, cudaStream_t s)
{
    return launch_exchange(d->pairs + (size_t)p * d->n_pairs, d->n_pairs, d->row_bytes, s);
}

}  // namespace

extern "C" {

lbm_status lbm_decomp_plan(int32_t ny, int32_t jc, int32_t hh, int32_t n_ranks, int32_t *row_start)
{
    return plan_split(ny, jc, hh, n_ranks, row_start, true);
}

lbm_status lbm_decomp_create(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                             const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads, int32_t n_ranks,
                             const int32_t *row_start, void *stream, const lbm_allocator *allocator,
                             lbm_decomp **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !lattice || !material) return fail(LBM_ERR_ARG, "grid, lattice and material are required");
    if (n_ranks < 1) return fail(LBM_ERR_ARG, "n_ranks must be >= 1");
    if (n_loads < 0 || (n_loads > 0 && !loads)) return fail(LBM_ERR_ARG, "bad loads array");
    for (int e = 0; e < 4; ++e)
        if (grid->edge[e] < LBM_EDGE_FREE || grid->edge[e] > LBM_EDGE_PERIODIC) return fail(LBM_ERR_ARG, "unknown edge kind");
    const int ny = grid->ny;
    const bool line_ok = lattice->velocity_set != LBM_D2Q9;   // a boundary on the crack line (D2Q5 only)
    const bool has_crack = crack && crack->mode != LBM_CRACK_NONE;
    int32_t jc = -1, hh = 0;
    if (has_crack) {
        const double yj = crack->y / grid->dh;
        if (!std::isfinite(yj) || std::fabs(yj - std::nearbyint(yj)) > 1e-9)
            return fail(LBM_ERR_ARG, "the crack line y must be a multiple of dh (between two rows)");
        jc = (int32_t)std::nearbyint(yj);
        hh = lattice->bc_mode != LBM_BC_BOUNCEBACK ? 3 : 1;
    }
    std::vector<int32_t> rs((size_t)n_ranks + 1);
    if (row_start) {
        std::copy(row_start, row_start + n_ranks + 1, rs.begin());
        if (!valid_split(ny, jc, hh, n_ranks, rs.data(), line_ok))
            return fail(LBM_ERR_ARG, line_ok ? "row_start must run from 0 to ny in slabs of >= 2 rows; a boundary may cut the crack rows only on the crack line"
                                             : "row_start must run from 0 to ny in slabs of >= 2 rows; a D2Q9 boundary may not cut the crack rows");
    } else {
        lbm_status rc = plan_split(ny, jc, hh, n_ranks, rs.data(), line_ok);
        if (rc != LBM_OK) return rc;
    }

    lbm_decomp *d = new (std::nothrow) lbm_decomp;
    if (!d) return fail(LBM_ERR_OOM, "host allocation failed");
    d->row_start = rs;
    d->crack_rank = -1;
    d->batch = nullptr;
    d->pairs = nullptr;
    d->n_pairs = 0;
    d->nx = grid->nx;
    d->ny = ny;
    d->stream = (cudaStream_t)stream;
    d->cap = nullptr;
    d->custom_alloc = allocator && allocator->alloc && allocator->release;
    if (d->custom_alloc) d->alloc = *allocator;
    const bool periodic_y = grid->edge[LBM_BOTTOM] == LBM_EDGE_PERIODIC;

    for (int r = 0; r < n_ranks; ++r) {
        const int32_t j0 = rs[(size_t)r], j1 = rs[(size_t)r + 1];
        lbm_grid g = *grid;
        g.ny = j1 - j0;
        if (n_ranks > 1) {
            if (r > 0 || periodic_y) g.edge[LBM_BOTTOM] = EDGE_HALO;
            if (r < n_ranks - 1 || periodic_y) g.edge[LBM_TOP] = EDGE_HALO;
        }
        lbm_crack c;
        std::memset(&c, 0, sizeof c);
        // the crack line inside the slab, or on one of its inner boundaries
        const bool mine = has_crack && ((jc > j0 && jc < j1) || (jc == j0 && r > 0) || (jc == j1 && r < n_ranks - 1));
        if (mine) {
            c = *crack;
            c.y = crack->y - (double)j0 * grid->dh;
            if (d->crack_rank < 0) d->crack_rank = r;
        }
        std::vector<lbm_loading> L;
        for (int q = 0; q < n_loads; ++q) {
            const int e = loads[q].edge;
            if ((e == LBM_BOTTOM && g.edge[e] == EDGE_HALO) || (e == LBM_TOP && g.edge[e] == EDGE_HALO)) continue;
            L.push_back(loads[q]);
        }
        lbm_handle *h = nullptr;
        lbm_status rc = create_impl(&g, lattice, material, mine ? &c : nullptr, L.empty() ? nullptr : L.data(),
                                    (int32_t)L.size(), stream, allocator, true, &h);
        if (rc != LBM_OK) {
            free_decomp(d);
            return rc;
        }
        d->slabs.push_back(h);
    }
    if (has_crack && d->crack_rank < 0) {
        free_decomp(d);
        return fail(LBM_ERR_ARG, "the crack line lies on no slab's interior");
    }
    d->esize = d->slabs[0]->esize;
    d->row_bytes = d->slabs[0]->pitch * (int64_t)d->esize;
    if (lattice->storage == LBM_F32_WD_F16) {
        // the scale the undivided lattice takes: the smallest over the slabs
        double scale = 0.0;
        for (lbm_handle *h : d->slabs) scale = scale == 0.0 ? h->wd_scale : std::min(scale, h->wd_scale);
        for (lbm_handle *h : d->slabs) {
            lbm_status rc = lbm_set_wd_scale(h, scale);
            if (rc != LBM_OK) {
                free_decomp(d);
                return rc;
            }
        }
    }
    lbm_status rc = lbm_batch_create(d->slabs.data(), n_ranks, 0, allocator, &d->batch);
    if (rc != LBM_OK) {
        free_decomp(d);
        return rc;
    }
    // halo pairs: boundary r between slabs r-1 and r (and the wrap-around)
    std::vector<RowCopy> pairs;
    for (int p = 0; p < 2; ++p) {
        auto link = [&](int lo, int hi) {
            const lbm_handle *a = d->slabs[(size_t)lo], *b = d->slabs[(size_t)hi];
            RowCopy up, down;
            up.src = row_ptr(a, p, a->grid.ny - 1, d->esize);   // top row of the lower slab
            up.dst = row_ptr(b, p, -1, d->esize);                // halo below the upper slab
            down.src = row_ptr(b, p, 0, d->esize);               // bottom row of the upper slab
            down.dst = row_ptr(a, p, a->grid.ny, d->esize);      // halo above the lower slab
            pairs.push_back(up);
            pairs.push_back(down);
        };
        for (int r = 1; r < n_ranks; ++r) link(r - 1, r);
        if (n_ranks > 1 && periodic_y) link(n_ranks - 1, 0);
    }
    d->n_pairs = (int)(pairs.size() / 2);
    if (d->n_pairs > 0) {
        const size_t bytes = pairs.size() * sizeof(RowCopy);
        if (d->custom_alloc) d->pairs = static_cast<RowCopy *>(d->alloc.alloc(bytes, d->alloc.ctx));
        else if (cudaMalloc(&d->pairs, bytes) != cudaSuccess) d->pairs = nullptr;
        if (!d->pairs) {
            free_decomp(d);
            return fail(LBM_ERR_OOM, "device allocation failed");
        }
        cudaError_t e = cudaMemcpyAsync(d->pairs, pairs.data(), bytes, cudaMemcpyHostToDevice, d->stream);
        if (e == cudaSuccess) e = exchange(d, batch_parity(d->batch), d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "uploading the halo table");
            free_decomp(d);
            return rc;
        }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "creating the capture stream");
        free_decomp(d);
        return rc;
    }
    *out = d;
    clear_error();
    return LBM_OK;
}

lbm_status lbm_decomp_step(lbm_decomp *d, int64_t n)
{
    lbm::NvtxRange nvtx_("lbm_decomp_step");
    if (!d) return fail(LBM_ERR_ARG, "decomposition is NULL");
    if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
    lbm_status rc = batch_check(d->batch);
    if (rc != LBM_OK) return rc;
    int par = batch_parity(d->batch);
    rc = run_chunks(d->graph, 0, d->stream, d->cap, n, par, [&](int p, cudaStream_t s) {
        cudaError_t e = batch_enqueue(d->batch, p, s);
        if (e != cudaSuccess) return e;
        return exchange(d, p ^ 1, s);   // the step wrote buffer p ^ 1
    });
    batch_mark_stepped(d->batch, par, n);
    return rc;
}

lbm_status lbm_decomp_fields(lbm_decomp *d, int32_t which, void *dst, int32_t dst_on_device, int32_t dtype)
{
    if (!d || !dst) return fail(LBM_ERR_ARG, "decomposition or dst is NULL");
    for (size_t r = 0; r < d->slabs.size(); ++r) {
        char *part = static_cast<char *>(dst) + (size_t)d->row_start[r] * (size_t)d->nx * d->esize;
        lbm_status rc = lbm_fields(d->slabs[r], which, part, dst_on_device, dtype);
        if (rc != LBM_OK) return rc;
    }
    return LBM_OK;
}

lbm_status lbm_decomp_set_fields(lbm_decomp *d, int32_t which, const void *src, int32_t src_on_device, int32_t dtype)
{
    if (!d || !src) return fail(LBM_ERR_ARG, "decomposition or src is NULL");
    for (size_t r = 0; r < d->slabs.size(); ++r) {
        const char *part = static_cast<const char *>(src) + (size_t)d->row_start[r] * (size_t)d->nx * d->esize;
        lbm_status rc = lbm_set_fields(d->slabs[r], which, part, src_on_device, dtype);
        if (rc != LBM_OK) return rc;
    }
    if (which == LBM_FIELD_W) LBM_CUDA(exchange(d, batch_parity(d->batch), d->stream));
    return LBM_OK;
}

lbm_status lbm_decomp_rank(const lbm_decomp *d, int32_t rank, lbm_handle **slab, int32_t *row0, int32_t *rows)
{
    if (!d) return fail(LBM_ERR_ARG, "decomposition is NULL");
    if (rank < 0 || rank >= (int32_t)d->slabs.size()) return fail(LBM_ERR_ARG, "rank out of range");
    if (slab) *slab = d->slabs[(size_t)rank];
    if (row0) *row0 = d->row_start[(size_t)rank];
    if (rows) *rows = d->row_start[(size_t)rank + 1] - d->row_start[(size_t)rank];
    return LBM_OK;
}

lbm_status lbm_decomp_info(const lbm_decomp *d, int32_t *n_ranks, int32_t *crack_rank)
{
    if (!d) return fail(LBM_ERR_ARG, "decomposition is NULL");
    if (n_ranks) *n_ranks = (int32_t)d->slabs.size();
    if (crack_rank) *crack_rank = d->crack_rank;
    return LBM_OK;
}

void lbm_decomp_destroy(lbm_decomp *d)
{
    if (!d) return;
    cudaStreamSynchronize(d->stream);
    free_decomp(d);
}

// ------------------------------------------ one slab per process (or device)

lbm_status lbm_slab_create(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                           const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads, int32_t row0,
                           int32_t rows, void *stream, const lbm_allocator *allocator, lbm_handle **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !lattice || !material) return fail(LBM_ERR_ARG, "grid, lattice and material are required");
    if (n_loads < 0 || (n_loads > 0 && !loads)) return fail(LBM_ERR_ARG, "bad loads array");
    for (int e = 0; e < 4; ++e)
        if (grid->edge[e] < LBM_EDGE_FREE || grid->edge[e] > LBM_EDGE_PERIODIC) return fail(LBM_ERR_ARG, "unknown edge kind");
    const int32_t ny = grid->ny, r1 = row0 + rows;
    if (row0 < 0 || rows < 2 || r1 > ny) return fail(LBM_ERR_ARG, "the slab must be >= 2 rows inside [0, ny)");
    const bool has_crack = crack && crack->mode != LBM_CRACK_NONE;
    int32_t jc = -1, hh = 0;
    if (has_crack) {
        const double yj = crack->y / grid->dh;
        if (!std::isfinite(yj) || std::fabs(yj - std::nearbyint(yj)) > 1e-9)
            return fail(LBM_ERR_ARG, "the crack line y must be a multiple of dh (between two rows)");
        jc = (int32_t)std::nearbyint(yj);
        hh = lattice->bc_mode != LBM_BC_BOUNCEBACK ? 3 : 1;
    }
    // this slab's side of each inner boundary (the neighbour checks its own)
    const bool line_ok = lattice->velocity_set != LBM_D2Q9;
    if ((row0 > 0 && !boundary_ok(row0, hh, rows, jc, hh, line_ok)) ||
        (r1 < ny && !boundary_ok(r1, rows, hh, jc, hh, line_ok)))
        return fail(LBM_ERR_ARG, line_ok ? "a slab boundary may cut the crack rows only on the crack line"
                                         : "a D2Q9 slab boundary may not cut the crack rows");
    const bool periodic_y = grid->edge[LBM_BOTTOM] == LBM_EDGE_PERIODIC;
    lbm_grid g = *grid;
    g.ny = rows;
    if (row0 > 0 || periodic_y) g.edge[LBM_BOTTOM] = EDGE_HALO;
    if (r1 < ny || periodic_y) g.edge[LBM_TOP] = EDGE_HALO;
    lbm_crack c;
    std::memset(&c, 0, sizeof c);
    const bool mine = has_crack && ((jc > row0 && jc < r1) || (jc == row0 && row0 > 0) || (jc == r1 && r1 < ny));
    if (mine) {
        c = *crack;
        c.y = crack->y - (double)row0 * grid->dh;
    }
    std::vector<lbm_loading> L;
    for (int q = 0; q < n_loads; ++q) {
        const int e = loads[q].edge;
        if ((e == LBM_BOTTOM || e == LBM_TOP) && g.edge[e] == EDGE_HALO) continue;
        L.push_back(loads[q]);
    }
    lbm_handle *h = nullptr;
    lbm_status rc = create_impl(&g, lattice, material, mine ? &c : nullptr, L.empty() ? nullptr : L.data(),
                                (int32_t)L.size(), stream, allocator, true, &h);
    if (rc != LBM_OK) return rc;
    if (lattice->storage == LBM_F32_WD_F16) {
        // every slab takes the scale of the undivided lattice
        rc = lbm_set_wd_scale(h, fp16_wd_scale(grid, loads, n_loads));
        if (rc != LBM_OK) {
            lbm_destroy(h);
            return rc;
        }
    }
    *out = h;
    clear_error();
    return LBM_OK;
}

lbm_status lbm_slab_export(lbm_handle *h, int32_t side, void *dst, int32_t dst_on_device)
{
    lbm::NvtxRange nvtx_("lbm_slab_export");
    if (!h || !dst) return fail(LBM_ERR_ARG, "handle or dst is NULL");
    if (side != 0 && side != 1) return fail(LBM_ERR_ARG, "side must be 0 (bottom row) or 1 (top row)");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    const int j = side == 0 ? 0 : h->grid.ny - 1;
    const char *src = static_cast<const char *>(h->w[h->parity]) + (int64_t)j * h->pitch * (int64_t)h->esize;
    const size_t bytes = (size_t)h->grid.nx * h->esize;
    LBM_CUDA(cudaMemcpyAsync(dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             h->stream));
    if (!dst_on_device) LBM_CUDA(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_slab_import(lbm_handle *h, int32_t side, const void *src, int32_t src_on_device)
{
    lbm::NvtxRange nvtx_("lbm_slab_import");
    if (!h || !src) return fail(LBM_ERR_ARG, "handle or src is NULL");
    if (side != 0 && side != 1) return fail(LBM_ERR_ARG, "side must be 0 (below row 0) or 1 (above the top row)");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (h->grid.edge[side == 0 ? LBM_BOTTOM : LBM_TOP] != EDGE_HALO)
        return fail(LBM_ERR_ARG, "that side of the slab is an outer edge, not a halo");
    const int j = side == 0 ? -1 : h->grid.ny;
    char *dst = static_cast<char *>(h->w[h->parity]) + (int64_t)j * h->pitch * (int64_t)h->esize;
    const size_t bytes = (size_t)h->grid.nx * h->esize;
    LBM_CUDA(cudaMemcpyAsync(dst, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             h->stream));
    if (!src_on_device) LBM_CUDA(cudaStreamSynchronize(h->stream));   // a pageable source may be reused
    return LBM_OK;
}

}  // extern "C"
