// lbm_tape.cu -- host runtime behind include/lbm_adjoint.h: the recording
// forward run (step kernel with sensor and cut-schedule recording), state
// snapshots every k steps, and the reverse sweep of the adjoint kernel, all
// replayed as CUDA graphs of 64-launch chunks on the handle's stream.
#include "lbm_adjoint.h"
#include "lbm_host.h"

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

using namespace lbm;
using namespace lbm::host;

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct lbm_tape {
    lbm_handle *h;
    int32_t ns;
    int64_t T;
    int32_t every;        // snapshot interval (0: keep the misfits of all steps)
    int64_t ring;         // rows of the misfit buffer
    int64_t n_ckpt;
    int32_t slots;        // partial sums per (step, edge)
    int32_t units_cap;
    lbm_allocator alloc;
    bool custom_alloc;
    void *block;
    size_t block_bytes;
    // device memory
    int32_t *s_i, *s_j, *s_off, *s_ent;
    double *target, *resid, *loss_acc, *loss, *part, *grad;
    int32_t *i_first, *i_last;
    int64_t *n0, *cnt;
    void *m[2], *a;       // adjoint planes, element (0, 0)
    void *mbase[2], *abase;
    void *dense;          // 2 x ny x nx staging for the field gradients
    char *ck;             // snapshots
    size_t ck_bytes, ck_w, ck_wd, ck_st, ck_cut;
    // host state
    std::vector<int32_t> sens;       // (i, j) pairs
    std::vector<int32_t> off_h, ent_h;
    std::vector<int> ck_pending;
    int recorded;
    int64_t rec_gen;
    int64_t cnt_init;
    ChunkGraph g_rec[2];  // recording steps without / with loss accumulation
    ChunkGraph g_adj;
    cudaStream_t cap;
};

namespace {

RecArgs rec_args(const lbm_tape *t, int acc_loss)
{
    RecArgs r;
    r.s_off = t->s_off;
    r.s_ent = t->s_ent;
    r.s_i = t->s_i;
    r.s_j = t->s_j;
    r.target = t->target;
    r.resid = t->resid;
    r.loss = t->loss_acc;
    r.i_first = t->i_first;
    r.i_last = t->i_last;
    r.n0 = t->n0;
    r.n_steps = t->T;
    r.ring = t->ring;
    r.ns = t->ns;
    r.acc_loss = acc_loss;
    return r;
}

template <typename T>
void make_adj_args(const lbm_tape *t, int par, AdjArgs<T> &a)
{
    const lbm_handle *h = t->h;
    a.w_in = static_cast<const T *>(t->m[par]);
    a.w_out = static_cast<T *>(t->m[par ^ 1]);
    a.wd = static_cast<T *>(t->a);
    a.wd_scale = (T)1;
    a.wd_inv = (T)1;
    a.pitch = h->pitch;
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.ncb = h->ncb;
    a.crack_band = h->crack_band;
    for (int e = 0; e < 4; ++e) a.edge[e] = h->grid.edge[e];
    a.g = (T)h->g;
    a.dt = (T)h->grid.dt;
    a.jc = h->jc;
    a.macro = h->cp.macro;
    a.pad0 = 0;
    a.i_first = t->i_first;
    a.ns = t->ns;
    a.units = h->units;
    a.i_last = t->i_last;
    a.cnt_in = t->cnt + par;
    a.cnt_out = t->cnt + (par ^ 1);
    a.n_steps = t->T;
    a.ring = t->ring;
    a.s_off = t->s_off;
    a.s_ent = t->s_ent;
    a.s_i = t->s_i;
    a.s_j = t->s_j;
    a.resid = t->resid;
    a.part = t->part;
    a.err = h->err;
    a.slots = t->slots;
    a.pad = 0;
}

// n recording steps of the handle from its current parity.
lbm_status record_steps(lbm_tape *t, int64_t n, int acc_loss)
{
    lbm_handle *h = t->h;
    const RecArgs r = rec_args(t, acc_loss);
    int par = h->parity;
    lbm_status rc;
    if (h->esize == 8) {
        rc = run_chunks(t->g_rec[acc_loss], h->gen, h->stream, t->cap, n, par, [&](int p, cudaStream_t s) {
            StepArgs<double, double> a;
            make_step_args(h, p, a);
            a.k_cta = use_k_cta(h) ? 1 : 0;
            return launch_step_rec<double>(a, r, h->n_bands, s);
        });
    } else {
        rc = run_chunks(t->g_rec[acc_loss], h->gen, h->stream, t->cap, n, par, [&](int p, cudaStream_t s) {
            StepArgs<float, float> a;
            make_step_args(h, p, a);
            a.k_cta = use_k_cta(h) ? 1 : 0;
            return launch_step_rec<float>(a, r, h->n_bands, s);
        });
    }
    h->parity = par;
    if (n > 0 && h->cp.mode != CRACK_NONE) h->pending = true;
    return rc;
}

// n transposed steps from adjoint parity *apar.
lbm_status adjoint_steps(lbm_tape *t, int64_t n, int &apar)
{
    lbm_handle *h = t->h;
    if (h->esize == 8)
        return run_chunks(t->g_adj, h->gen, h->stream, t->cap, n, apar, [&](int p, cudaStream_t s) {
            AdjArgs<double> a;
            make_adj_args(t, p, a);
            return launch_adjoint<double>(a, h->n_bands, s);
        });
    return run_chunks(t->g_adj, h->gen, h->stream, t->cap, n, apar, [&](int p, cudaStream_t s) {
        AdjArgs<float> a;
        make_adj_args(t, p, a);
        return launch_adjoint<float>(a, h->n_bands, s);
    });
}

// Copy the handle's state (fields of the current parity with their pads,
// crack state, crack row of the cut mask) into snapshot k, or back.
lbm_status snapshot(lbm_tape *t, int64_t k, bool save)
{
    lbm_handle *h = t->h;
    char *c = t->ck + (size_t)k * t->ck_bytes;
    cudaStream_t s = h->stream;
    const cudaMemcpyKind D2D = cudaMemcpyDeviceToDevice;
    char *crow = reinterpret_cast<char *>(h->cut_v + (size_t)(h->jc > 0 ? h->jc - 1 : 0) * h->words);
    const size_t cut_bytes = (size_t)h->words * 4;
    if (save) {
        LBM_CUDA(cudaMemcpyAsync(c + t->ck_w, h->wbase[h->parity], h->plane_bytes, D2D, s));
        LBM_CUDA(cudaMemcpyAsync(c + t->ck_wd, h->wdbase, h->plane_d_bytes, D2D, s));
        LBM_CUDA(cudaMemcpyAsync(c + t->ck_st, h->st + h->parity, sizeof(CrackState), D2D, s));
        if (h->cp.mode != CRACK_NONE) LBM_CUDA(cudaMemcpyAsync(c + t->ck_cut, crow, cut_bytes, D2D, s));
        t->ck_pending[(size_t)k] = h->pending ? 1 : 0;
    } else {
        LBM_CUDA(cudaMemcpyAsync(h->wbase[h->parity], c + t->ck_w, h->plane_bytes, D2D, s));
        LBM_CUDA(cudaMemcpyAsync(h->wdbase, c + t->ck_wd, h->plane_d_bytes, D2D, s));
        LBM_CUDA(cudaMemcpyAsync(h->st + h->parity, c + t->ck_st, sizeof(CrackState), D2D, s));
        if (h->cp.mode != CRACK_NONE) LBM_CUDA(cudaMemcpyAsync(crow, c + t->ck_cut, cut_bytes, D2D, s));
        h->pending = t->ck_pending[(size_t)k] != 0;
    }
    return LBM_OK;
}

// Sensor lists per unit of the handle's current partition.
lbm_status upload_sensor_lists(lbm_tape *t)
{
    lbm_handle *h = t->h;
    const std::vector<Unit> &U = *h->units_h;
    const int n_units = (int)U.size() * h->ncb;
    if (n_units + 1 > t->units_cap) return fail(LBM_ERR_STATE, "the launch shape changed beyond the tape's tables");
    const int cols = kThreads * (int)(16 / h->esize);
    std::vector<int> unit_of((size_t)t->ns);
    std::vector<int32_t> &off = t->off_h, &ent = t->ent_h;
    off.assign((size_t)n_units + 1, 0);
    ent.assign((size_t)t->ns, 0);
    for (int k = 0; k < t->ns; ++k) {
        const int i = t->sens[2 * (size_t)k], j = t->sens[2 * (size_t)k + 1];
        int b = 0;
        while (b < (int)U.size() && !(U[(size_t)b].j0 <= j && j < U[(size_t)b].j1)) ++b;
        if (b == (int)U.size()) return fail(LBM_ERR_STATE, "a sensor row lies in no band");
        unit_of[(size_t)k] = b * h->ncb + i / cols;
        off[(size_t)unit_of[(size_t)k] + 1] += 1;
    }
    for (int u = 0; u < n_units; ++u) off[(size_t)u + 1] += off[(size_t)u];
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int k = 0; k < t->ns; ++k) ent[(size_t)fill[(size_t)unit_of[(size_t)k]]++] = k;
    LBM_CUDA(cudaMemcpyAsync(t->s_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice, h->stream));
    if (t->ns > 0) LBM_CUDA(cudaMemcpyAsync(t->s_ent, ent.data(), ent.size() * 4, cudaMemcpyHostToDevice, h->stream));
    return LBM_OK;
}

void free_tape(lbm_tape *t)
{
    t->g_rec[0].reset();
    t->g_rec[1].reset();
    t->g_adj.reset();
    if (t->cap) cudaStreamDestroy(t->cap);
    if (t->block) {
        if (t->custom_alloc) t->alloc.release(t->block, t->alloc.ctx);
        else cudaFree(t->block);
    }
    delete t;
}

}  // namespace

extern "C" {

lbm_status lbm_tape_create(lbm_handle *h, const int32_t *sensors, int32_t n_sens, int64_t n_steps,
                           int32_t checkpoint_every, const lbm_allocator *allocator, lbm_tape **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (h->lat.storage != LBM_F64 && h->lat.storage != LBM_F32)
        return fail(LBM_ERR_ARG, "the adjoint needs LBM_F64 or LBM_F32 storage");
    if (h->edge_macro) return fail(LBM_ERR_ARG, "the adjoint has no macroscopic rule on the outer edges");
    if (h->q != 5) return fail(LBM_ERR_ARG, "the adjoint is built for D2Q5 only");
    if (h->line) return fail(LBM_ERR_ARG, "the adjoint is built for cracks along +x");
    if (h->grid.edge[LBM_BOTTOM] == EDGE_HALO || h->grid.edge[LBM_TOP] == EDGE_HALO)
        return fail(LBM_ERR_ARG, "the adjoint is not built for row slabs");
    if (n_sens < 0 || (n_sens > 0 && !sensors)) return fail(LBM_ERR_ARG, "bad sensor array");
    if (n_steps < 1 || n_steps > ((int64_t)1 << 31)) return fail(LBM_ERR_ARG, "n_steps must lie in [1, 2^31]");
    if (checkpoint_every < 0) return fail(LBM_ERR_ARG, "checkpoint_every must be >= 0");
    const int nx = h->grid.nx, ny = h->grid.ny;
    for (int32_t k = 0; k < n_sens; ++k)
        if (sensors[2 * k] < 0 || sensors[2 * k] >= nx || sensors[2 * k + 1] < 0 || sensors[2 * k + 1] >= ny)
            return fail(LBM_ERR_ARG, "a sensor lies outside the lattice");

    lbm_tape *t = new (std::nothrow) lbm_tape;
    if (!t) return fail(LBM_ERR_OOM, "host allocation failed");
    t->h = h;
    t->ns = n_sens;
    t->T = n_steps;
    t->every = checkpoint_every >= n_steps ? 0 : checkpoint_every;
    t->ring = t->every > 0 ? t->every : n_steps;
    t->n_ckpt = t->every > 0 ? (n_steps + t->every - 1) / t->every + 1 : 0;
    t->slots = std::max(h->ncb, h->n_bands);
    t->units_cap = ny * h->ncb + 1;
    t->custom_alloc = allocator && allocator->alloc && allocator->release;
    if (t->custom_alloc) t->alloc = *allocator;
    t->block = nullptr;
    t->cap = nullptr;
    t->recorded = 0;
    t->rec_gen = -1;
    t->cnt_init = n_steps;
    t->sens.assign(sensors, sensors + 2 * (size_t)n_sens);
    t->ck_pending.assign((size_t)t->n_ckpt, 0);

    const size_t ns = (size_t)n_sens, T = (size_t)n_steps;
    const size_t dense = 2 * (size_t)nx * ny * h->esize;
    t->ck_w = 0;
    t->ck_wd = align256(h->plane_bytes);
    t->ck_st = t->ck_wd + align256(h->plane_d_bytes);
    t->ck_cut = t->ck_st + align256(sizeof(CrackState));
    t->ck_bytes = t->ck_cut + align256((size_t)h->words * 4);
    size_t off = 0;
    const size_t o_si = off; off = align256(off + ns * 4);
    const size_t o_sj = off; off = align256(off + ns * 4);
    const size_t o_so = off; off = align256(off + (size_t)t->units_cap * 4);
    const size_t o_se = off; off = align256(off + ns * 4);
    const size_t o_tg = off; off = align256(off + T * ns * 8);
    const size_t o_rs = off; off = align256(off + (size_t)t->ring * ns * 8);
    const size_t o_la = off; off = align256(off + ns * 8);
    const size_t o_lo = off; off = align256(off + 8);
    const size_t o_pt = off; off = align256(off + T * 4 * (size_t)t->slots * 8);
    const size_t o_gr = off; off = align256(off + 4 * T * 8);
    const size_t o_if = off; off = align256(off + T * 4);
    const size_t o_il = off; off = align256(off + T * 4);
    const size_t o_n0 = off; off = align256(off + 8);
    const size_t o_ct = off; off = align256(off + 16);
    const size_t o_m0 = off; off = align256(off + h->plane_bytes);
    const size_t o_m1 = off; off = align256(off + h->plane_bytes);
    const size_t o_a = off; off = align256(off + h->plane_bytes);
    const size_t o_dn = off; off = align256(off + dense);
    const size_t o_ck = off; off = align256(off + (size_t)t->n_ckpt * t->ck_bytes);
    t->block_bytes = off;
    if (t->custom_alloc) t->block = t->alloc.alloc(off, t->alloc.ctx);
    else if (cudaMalloc(&t->block, off) != cudaSuccess) t->block = nullptr;
    if (!t->block) {
        free_tape(t);
        return fail(LBM_ERR_OOM, "device allocation failed");
    }
    char *b = static_cast<char *>(t->block);
    t->s_i = reinterpret_cast<int32_t *>(b + o_si);
    t->s_j = reinterpret_cast<int32_t *>(b + o_sj);
    t->s_off = reinterpret_cast<int32_t *>(b + o_so);
    t->s_ent = reinterpret_cast<int32_t *>(b + o_se);
    t->target = reinterpret_cast<double *>(b + o_tg);
    t->resid = reinterpret_cast<double *>(b + o_rs);
    t->loss_acc = reinterpret_cast<double *>(b + o_la);
    t->loss = reinterpret_cast<double *>(b + o_lo);
    t->part = reinterpret_cast<double *>(b + o_pt);
    t->grad = reinterpret_cast<double *>(b + o_gr);
    t->i_first = reinterpret_cast<int32_t *>(b + o_if);
    t->i_last = reinterpret_cast<int32_t *>(b + o_il);
    t->n0 = reinterpret_cast<int64_t *>(b + o_n0);
    t->cnt = reinterpret_cast<int64_t *>(b + o_ct);
    const size_t xoff = 128 / h->esize;
    const size_t origin = ((size_t)h->pitch + xoff) * h->esize;
    t->mbase[0] = b + o_m0;
    t->mbase[1] = b + o_m1;
    t->abase = b + o_a;
    t->m[0] = b + o_m0 + origin;
    t->m[1] = b + o_m1 + origin;
    t->a = b + o_a + origin;
    t->dense = b + o_dn;
    t->ck = b + o_ck;

    cudaStream_t s = h->stream;
    std::vector<int32_t> si(ns), sj(ns);
    for (size_t k = 0; k < ns; ++k) {
        si[k] = sensors[2 * k];
        sj[k] = sensors[2 * k + 1];
    }
    cudaError_t e = cudaMemsetAsync(t->block, 0, t->block_bytes, s);
    if (e == cudaSuccess && ns) e = cudaMemcpyAsync(t->s_i, si.data(), ns * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && ns) e = cudaMemcpyAsync(t->s_j, sj.data(), ns * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        lbm_status rc = cuda_fail(e, "initialising the tape");
        free_tape(t);
        return rc;
    }
    *out = t;
    clear_error();
    return LBM_OK;
}

lbm_status lbm_tape_forward(lbm_tape *t, const double *targets, int32_t targets_on_device, double *loss)
{
    lbm::NvtxRange nvtx_("lbm_tape_forward");
    if (!t) return fail(LBM_ERR_ARG, "tape is NULL");
    if (!targets && t->ns > 0) return fail(LBM_ERR_ARG, "targets is NULL");
    lbm_handle *h = t->h;
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (h->n_bands > t->slots) return fail(LBM_ERR_STATE, "the launch shape changed beyond the tape's tables");
    cudaStream_t s = h->stream;
    t->recorded = 0;
    lbm_status rc = upload_sensor_lists(t);
    if (rc != LBM_OK) return rc;
    const size_t tbytes = (size_t)t->T * (size_t)t->ns * 8;
    if (tbytes)
        LBM_CUDA(cudaMemcpyAsync(t->target, targets, tbytes,
                                 targets_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (t->ns) LBM_CUDA(cudaMemsetAsync(t->loss_acc, 0, (size_t)t->ns * 8, s));
    // the step count the recording starts from
    LBM_CUDA(cudaMemcpyAsync(t->n0, reinterpret_cast<const char *>(h->st + h->parity) + offsetof(CrackState, step), 8,
                             cudaMemcpyDeviceToDevice, s));
    if (t->every == 0) {
        rc = record_steps(t, t->T, 1);
        if (rc != LBM_OK) return rc;
    } else {
        int64_t seg = 0;
        for (int64_t t0 = 0; t0 < t->T; t0 += t->every, ++seg) {
            if ((rc = snapshot(t, seg, true)) != LBM_OK) return rc;
            if ((rc = record_steps(t, std::min<int64_t>(t->every, t->T - t0), 1)) != LBM_OK) return rc;
        }
        if ((rc = snapshot(t, seg, true)) != LBM_OK) return rc;
    }
    LBM_CUDA(launch_loss_sum(t->loss_acc, t->ns, t->loss, s));
    t->recorded = 1;
    t->rec_gen = h->gen;
    if (!targets_on_device) LBM_CUDA(cudaStreamSynchronize(s));   // pageable targets may be reused
    if (loss) {
        LBM_CUDA(cudaMemcpyAsync(loss, t->loss, 8, cudaMemcpyDeviceToHost, s));
        return check_sticky(h);
    }
    return LBM_OK;
}

lbm_status lbm_tape_loss_device(const lbm_tape *t, const double **loss)
{
    if (!t || !loss) return fail(LBM_ERR_ARG, "tape or loss is NULL");
    *loss = t->loss;
    return LBM_OK;
}

lbm_status lbm_tape_backward(lbm_tape *t, double *dL_dload, int32_t load_on_device, void *dL_dw0, void *dL_dwdot0,
                             int32_t fields_on_device, int32_t dtype)
{
    lbm::NvtxRange nvtx_("lbm_tape_backward");
    if (!t) return fail(LBM_ERR_ARG, "tape is NULL");
    lbm_handle *h = t->h;
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (!t->recorded) return fail(LBM_ERR_STATE, "no recording (call lbm_tape_forward first)");
    if (h->gen != t->rec_gen) return fail(LBM_ERR_STATE, "the handle's launch shape or loads changed since the recording");
    if ((dL_dw0 || dL_dwdot0) && dtype != (h->esize == 8 ? LBM_F64 : LBM_F32))
        return fail(LBM_ERR_ARG, "dtype must be LBM_F64 for F64 storage, LBM_F32 for F32");
    cudaStream_t s = h->stream;
    LBM_CUDA(cudaMemsetAsync(t->part, 0, (size_t)t->T * 4 * (size_t)t->slots * 8, s));
    LBM_CUDA(cudaMemsetAsync(t->mbase[0], 0, h->plane_bytes, s));
    LBM_CUDA(cudaMemsetAsync(t->mbase[1], 0, h->plane_bytes, s));
    LBM_CUDA(cudaMemsetAsync(t->abase, 0, h->plane_bytes, s));
    LBM_CUDA(cudaMemcpyAsync(t->cnt, &t->cnt_init, 8, cudaMemcpyHostToDevice, s));
    int apar = 0;
    lbm_status rc;
    if (t->every == 0) {
        // transposed steps T, T-1, ..., 0 (step T: the sources of the last state)
        if ((rc = adjoint_steps(t, t->T + 1, apar)) != LBM_OK) return rc;
    } else {
        const int64_t nseg = (t->T + t->every - 1) / t->every;
        for (int64_t seg = nseg - 1; seg >= 0; --seg) {
            const int64_t t0 = seg * t->every, t1 = std::min<int64_t>(t->T, t0 + t->every);
            if ((rc = snapshot(t, seg, false)) != LBM_OK) return rc;
            if ((rc = record_steps(t, t1 - t0, 0)) != LBM_OK) return rc;   // misfits of states t0+1 .. t1
            if ((rc = adjoint_steps(t, t1 - t0, apar)) != LBM_OK) return rc;   // transposed steps t1 .. t0+1
        }
        if ((rc = adjoint_steps(t, 1, apar)) != LBM_OK) return rc;   // transposed step 0
        if ((rc = snapshot(t, nseg, false)) != LBM_OK) return rc;    // back to the end of the run
    }
    int dir_mask = 0;
    for (int e = 0; e < 4; ++e)
        if (h->grid.edge[e] == LBM_EDGE_DIRICHLET) dir_mask |= 1 << e;
    LBM_CUDA(launch_grad_sum(t->part, t->T, t->slots, dir_mask, h->g, t->grad, s));
    const int nx = h->grid.nx, ny = h->grid.ny;
    const size_t nf = (size_t)nx * ny;
    if (dL_dw0 || dL_dwdot0) {
        char *dn = static_cast<char *>(t->dense);
        if (h->esize == 8)
            LBM_CUDA(launch_adjoint_out<double>(static_cast<const double *>(t->a), static_cast<const double *>(t->m[apar]),
                                                h->pitch, nx, ny, h->grid.dt, reinterpret_cast<double *>(dn),
                                                reinterpret_cast<double *>(dn) + nf, s));
        else
            LBM_CUDA(launch_adjoint_out<float>(static_cast<const float *>(t->a), static_cast<const float *>(t->m[apar]),
                                               h->pitch, nx, ny, (float)h->grid.dt, reinterpret_cast<float *>(dn),
                                               reinterpret_cast<float *>(dn) + nf, s));
        const cudaMemcpyKind kf = fields_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (dL_dw0) LBM_CUDA(cudaMemcpyAsync(dL_dw0, dn, nf * h->esize, kf, s));
        if (dL_dwdot0) LBM_CUDA(cudaMemcpyAsync(dL_dwdot0, dn + nf * h->esize, nf * h->esize, kf, s));
    }
    if (dL_dload)
        LBM_CUDA(cudaMemcpyAsync(dL_dload, t->grad, 4 * (size_t)t->T * 8,
                                 load_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    const bool host_out = (dL_dload && !load_on_device) || ((dL_dw0 || dL_dwdot0) && !fields_on_device);
    if (host_out) return check_sticky(h);
    return LBM_OK;
}

lbm_status lbm_tape_misfits(lbm_tape *t, double *dst, int32_t dst_on_device)
{
    if (!t || !dst) return fail(LBM_ERR_ARG, "tape or dst is NULL");
    if (!t->recorded) return fail(LBM_ERR_STATE, "no recording");
    if (t->every != 0) return fail(LBM_ERR_STATE, "a checkpointed tape keeps only one segment's misfits");
    lbm_handle *h = t->h;
    const size_t bytes = (size_t)t->T * (size_t)t->ns * 8;
    if (bytes)
        LBM_CUDA(cudaMemcpyAsync(dst, t->resid, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 h->stream));
    if (!dst_on_device) return check_sticky(h);
    return LBM_OK;
}

void lbm_tape_destroy(lbm_tape *t)
{
    if (!t) return;
    cudaStreamSynchronize(t->h->stream);
    free_tape(t);
}

lbm_status lbm_adjoint(lbm_handle *h, const int32_t *sensors, int32_t n_sens, int64_t n_steps, int32_t checkpoint_every,
                       const double *targets, int32_t targets_on_device, double *loss, double *dL_dload,
                       int32_t load_on_device, void *dL_dw0, void *dL_dwdot0, int32_t fields_on_device, int32_t dtype,
                       const lbm_allocator *allocator)
{
    lbm::NvtxRange nvtx_("lbm_adjoint");
    lbm_tape *t = nullptr;
    lbm_status rc = lbm_tape_create(h, sensors, n_sens, n_steps, checkpoint_every, allocator, &t);
    if (rc != LBM_OK) return rc;
    rc = lbm_tape_forward(t, targets, targets_on_device, loss);
    if (rc == LBM_OK) rc = lbm_tape_backward(t, dL_dload, load_on_device, dL_dw0, dL_dwdot0, fields_on_device, dtype);
    const std::string msg = rc == LBM_OK ? std::string() : std::string(last_error());
    lbm_tape_destroy(t);   // synchronises the handle's stream: the outputs are complete
    if (rc != LBM_OK) return fail(rc, msg);
    return LBM_OK;
}

}  // extern "C"
