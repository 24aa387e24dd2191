// lbm_api.cu -- host runtime behind the C ABI declared in include/lbm.h:
// validation, device memory layout, initial crack, the static band partition
// of the step kernel, CUDA-graph replay of step sequences, the deferred crack
// step before host reads, and the copy-out calls.
#include "lbm_host.h"

#include <type_traits>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

using namespace lbm;
using namespace lbm::host;

namespace lbm {
namespace host {

namespace {
thread_local std::string g_err;
}

lbm_status fail(lbm_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

lbm_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
}

void clear_error() { g_err.clear(); }

const char *last_error() { return g_err.c_str(); }

void ChunkGraph::reset()
{
    for (auto &lv : exec)
        for (auto &ex : lv) {
            if (ex) cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    gen = -1;
}

}  // namespace host
}  // namespace lbm

namespace {

constexpr int64_t kDefaultHistCap = 65536;

int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------ geometry of a crack in any direction
// Exact on the 2^-32 dh grid (128-bit cross products).

int64_t centre_q(int64_t i) { return (2 * i + 1) << (kQBits - 1); }

int orient_q(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy)
{
    const __int128 v = (__int128)(bx - ax) * (__int128)(cy - ay) - (__int128)(by - ay) * (__int128)(cx - ax);
    return (v > 0) - (v < 0);
}

bool within_q(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py)
{
    return px >= std::min(ax, bx) && px <= std::max(ax, bx) && py >= std::min(ay, by) && py <= std::max(ay, by);
}

// Do the closed segments p1p2 and q1q2 meet?
bool segments_meet_q(int64_t p1x, int64_t p1y, int64_t p2x, int64_t p2y, int64_t q1x, int64_t q1y, int64_t q2x,
                     int64_t q2y)
{
    const int a = orient_q(q1x, q1y, q2x, q2y, p1x, p1y), b = orient_q(q1x, q1y, q2x, q2y, p2x, p2y);
    const int c = orient_q(p1x, p1y, p2x, p2y, q1x, q1y), d = orient_q(p1x, p1y, p2x, p2y, q2x, q2y);
    if (a * b < 0 && c * d < 0) return true;
    return (a == 0 && within_q(q1x, q1y, q2x, q2y, p1x, p1y)) || (b == 0 && within_q(q1x, q1y, q2x, q2y, p2x, p2y)) ||
           (c == 0 && within_q(p1x, p1y, p2x, p2y, q1x, q1y)) || (d == 0 && within_q(p1x, p1y, p2x, p2y, q2x, q2y));
}

// Does the line through S and T pass through a site centre of the lattice?
// Along the axis of its larger extent each column (row) holds one candidate
// crossing; the sites next to it are tested exactly.
bool line_hits_a_centre(const LineSpec &L, int nx, int ny)
{
    const int64_t dx = L.tip_xq - L.start_xq, dy = L.tip_yq - L.start_yq;
    const bool by_col = (dx < 0 ? -dx : dx) >= (dy < 0 ? -dy : dy);
    const int n = by_col ? nx : ny, m = by_col ? ny : nx;
    for (int i = 0; i < n; ++i) {
        const double c = ((double)i + 0.5) * 4294967296.0;
        const double t = by_col ? (c - (double)L.start_xq) / (double)dx : (c - (double)L.start_yq) / (double)dy;
        const double o = (by_col ? (double)L.start_yq + t * (double)dy : (double)L.start_xq + t * (double)dx) / 4294967296.0;
        if (!(o > -2.0 && o < (double)m + 2.0)) continue;
        const int j0 = (int)std::floor(o - 0.5);
        for (int j = j0 - 1; j <= j0 + 2; ++j) {
            if (j < 0 || j >= m) continue;
            const int64_t cx = centre_q(by_col ? i : j), cy = centre_q(by_col ? j : i);
            if (orient_q(L.start_xq, L.start_yq, L.tip_xq, L.tip_yq, cx, cy) == 0) return true;
        }
    }
    return false;
}

// The initial crack: every H and V link the segment from the start to the
// tip meets, as [H mask | V mask] (ny rows of `words` words each).
std::vector<uint32_t> line_initial_masks(const LineSpec &L, int nx, int ny, int words)
{
    std::vector<uint32_t> m((size_t)2 * ny * words, 0u);
    const int64_t one = (int64_t)1 << kQBits, half = one / 2;
    const int64_t i0 = std::max<int64_t>(0, floor_div(std::min(L.start_xq, L.tip_xq) - 3 * half, one));
    const int64_t i1 = std::min<int64_t>(nx - 1, floor_div(std::max(L.start_xq, L.tip_xq) + half, one) + 1);
    const int64_t j0 = std::max<int64_t>(0, floor_div(std::min(L.start_yq, L.tip_yq) - 3 * half, one));
    const int64_t j1 = std::min<int64_t>(ny - 1, floor_div(std::max(L.start_yq, L.tip_yq) + half, one) + 1);
    const size_t vo = (size_t)ny * words;
    for (int64_t j = j0; j <= j1; ++j)
        for (int64_t i = i0; i <= i1; ++i) {
            const int64_t cx = centre_q(i), cy = centre_q(j);
            const size_t wi = (size_t)j * words + (size_t)(i >> 5);
            if (i + 1 < nx && segments_meet_q(cx, cy, centre_q(i + 1), cy, L.start_xq, L.start_yq, L.tip_xq, L.tip_yq))
                m[wi] |= 1u << (i & 31);
            if (j + 1 < ny && segments_meet_q(cx, cy, cx, centre_q(j + 1), L.start_xq, L.start_yq, L.tip_xq, L.tip_yq))
                m[vo + wi] |= 1u << (i & 31);
        }
    return m;
}

// The boundary points of the macroscopic rule on the faces of a crack in any
// direction (LineFace): every site within 1.5 spacings of the line (the
// sites next to a severed link lie within one), with the stencils of x_I
// and x_II along the line's normal and the weights of the quadratic with
// zero slope at the line.  A stencil with a corner outside the body is
// dropped (its value counts as 0) and the entry marked in `dropped`.
std::vector<LineFace> line_faces_table(const LineSpec &L, int nx, int ny, std::vector<uint8_t> *dropped = nullptr)
{
    const double sx = (double)L.start_xq * kTwoM32, sy = (double)L.start_yq * kTwoM32;
    const double cx = L.dir_x, cy = L.dir_y;
    auto dist = [&](double x, double y) { return -(x - sx) * cy + (y - sy) * cx; };
    std::vector<std::pair<int, int>> sites;
    const bool by_col = std::fabs(cx) >= std::fabs(cy);
    const int n = by_col ? nx : ny, m = by_col ? ny : nx;
    for (int l = 0; l < n; ++l) {
        const double across = by_col ? sy + ((l + 0.5) - sx) * cy / cx : sx + ((l + 0.5) - sy) * cx / cy;
        if (!(across > -4.0 && across < m + 4.0)) continue;
        const int k0 = (int)std::floor(across - 3.0);
        for (int k = k0; k <= k0 + 6; ++k) {
            if (k < 0 || k >= m) continue;
            const int i = by_col ? l : k, j = by_col ? k : l;
            if (std::fabs(dist(i + 0.5, j + 0.5)) < 1.5) sites.emplace_back(i, j);
        }
    }
    std::unordered_map<int64_t, int32_t> index;
    for (size_t q = 0; q < sites.size(); ++q) index[(int64_t)sites[q].second * nx + sites[q].first] = (int32_t)q;
    std::vector<LineFace> tab(sites.size());
    if (dropped) dropped->assign(sites.size(), 0);
    for (size_t q = 0; q < sites.size(); ++q) {
        LineFace &f = tab[q];
        std::memset(&f, 0, sizeof f);
        f.i = sites[q].first;
        f.j = sites[q].second;
        const double bx = f.i + 0.5, by = f.j + 0.5;
        const double d = dist(bx, by), side = d > 0.0 ? 1.0 : -1.0;
        const double nxv = -cy * side, nyv = cx * side;
        const double sB = std::fabs(d), sI = sB + 1.0, sII = sB + 2.0;
        const double qq = (sB * sB - sI * sI) / (sII * sII - sI * sI);
        const double coef[2] = {1.0 - qq, qq};
        int used = 0;
        for (int pt = 0; pt < 2; ++pt) {
            const double px = bx + (pt + 1) * nxv, py = by + (pt + 1) * nyv;
            const double gx = px - 0.5, gy = py - 0.5;
            const int i0 = (int)std::floor(gx), j0 = (int)std::floor(gy);
            const double tx = gx - i0, ty = gy - j0;
            int ci[4], cj[4];
            double wt[4];
            int nc = 0;
            bool inside = true;
            for (int dj = 0; dj <= 1; ++dj)
                for (int di = 0; di <= 1; ++di) {
                    const double wgt = (di ? tx : 1.0 - tx) * (dj ? ty : 1.0 - ty);
                    if (wgt == 0.0) continue;
                    const int ii = i0 + di, jj = j0 + dj;
                    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) inside = false;
                    ci[nc] = ii;
                    cj[nc] = jj;
                    wt[nc] = wgt;
                    ++nc;
                }
            if (!inside) {
                if (dropped) (*dropped)[q] = 1;
                f.flags |= lbm::FACE_DROPPED;
                continue;
            }
            for (int c = 0; c < nc; ++c) {
                f.ci[used] = ci[c];
                f.cj[used] = cj[c];
                f.a[used] = coef[pt] * wt[c];
                const auto it = index.find((int64_t)cj[c] * nx + ci[c]);
                f.cand[used] = it == index.end() ? -1 : it->second;
                ++used;
            }
        }
        for (int c = used; c < 8; ++c) {
            f.ci[c] = f.i;
            f.cj[c] = f.j;
            f.cand[c] = -1;
            f.a[c] = 0.0;
        }
        for (int c = 0; c < 8; ++c) f.af[c] = (float)f.a[c];
    }
    return tab;
}

// The chunked face solve's tables (FaceChunk): chunks of kFaceChunk
// consecutive table entries with the transitive closure of their coupled
// corners, sorted by level.  Returns false (leaving the one-CTA solve in
// use) when the coupling has a cycle through more than one entry, is deeper
// than kFaceLevels, or a chunk's closure exceeds kFaceItemsMax.
bool line_face_chunks(const std::vector<LineFace> &tab, std::vector<lbm::FaceChunk> &chunks,
                      std::vector<lbm::FaceItem> &items)
{
    using lbm::kFaceChunk;
    using lbm::kFaceItemsMax;
    using lbm::kFaceLevels;
    const int n = (int)tab.size();
    auto corners = [&](int e, std::vector<int> &out) {
        out.clear();
        for (int k = 0; k < 8; ++k)
            if (tab[e].a[k] != 0.0 && tab[e].cand[k] >= 0 && tab[e].cand[k] != e) out.push_back(tab[e].cand[k]);
    };
    // levels by depth-first search (0: unvisited, 1: on the stack, 2: done)
    std::vector<int> level(n, 0), state(n, 0);
    std::vector<int> cs;
    for (int r = 0; r < n; ++r) {
        if (state[r]) continue;
        std::vector<std::pair<int, int>> stack{{r, 0}};
        state[r] = 1;
        while (!stack.empty()) {
            const int e = stack.back().first;
            corners(e, cs);
            int &next = stack.back().second;
            if (next < (int)cs.size()) {
                const int m = cs[next++];
                if (state[m] == 1) return false;   // a cycle
                if (state[m] == 0) {
                    state[m] = 1;
                    stack.push_back({m, 0});
                }
                continue;
            }
            int lv = 0;
            for (int m : cs) lv = std::max(lv, level[m] + 1);
            if (lv >= kFaceLevels) return false;
            level[e] = lv;
            state[e] = 2;
            stack.pop_back();
        }
    }
    chunks.clear();
    items.clear();
    std::vector<int> local(n, -1);
    for (int lo = 0; lo < n; lo += kFaceChunk) {
        const int hi = std::min(n, lo + kFaceChunk);
        std::vector<int> clo;
        for (int e = lo; e < hi; ++e) {
            local[e] = 0;
            clo.push_back(e);
        }
        for (size_t q = 0; q < clo.size(); ++q) {
            corners(clo[q], cs);
            for (int m : cs)
                if (local[m] < 0) {
                    local[m] = 0;
                    clo.push_back(m);
                }
        }
        if ((int)clo.size() > kFaceItemsMax) return false;
        std::stable_sort(clo.begin(), clo.end(), [&](int x, int y) {
            return level[x] != level[y] ? level[x] < level[y] : x < y;
        });
        for (size_t q = 0; q < clo.size(); ++q) local[clo[q]] = (int)q;
        lbm::FaceChunk c;
        std::memset(&c, 0, sizeof c);
        c.off = (int32_t)items.size();
        c.n = (int32_t)clo.size();
        c.own_lo = lo;
        c.own_hi = hi;
        for (int L = 0; L <= kFaceLevels; ++L) {
            int q = 0;
            while (q < (int)clo.size() && level[clo[q]] < L) ++q;
            c.lv[L] = q;
        }
        for (int e : clo) {
            lbm::FaceItem it;
            std::memset(&it, 0, sizeof it);
            it.rec = tab[e];
            it.f = e;
            for (int k = 0; k < 8; ++k) {
                const int m = tab[e].cand[k];
                it.kl[k] = (int16_t)((tab[e].a[k] != 0.0 && m >= 0) ? local[m] : -1);
            }
            items.push_back(it);
        }
        chunks.push_back(c);
        for (int e : clo) local[e] = -1;
    }
    return true;
}

}  // namespace


namespace {


template <typename T, typename D>
cudaError_t enqueue_step_t(const lbm_handle *h, int par, cudaStream_t s)
{
    StepArgs<T, D> a;
    make_step_args(h, par, a);
    if constexpr (!std::is_same<D, Lf>::value) {   // a crack in any direction has no leapfrog storage
        if (h->line) {
            cudaError_t e;
            {
                lbm::NvtxRange r("K1 line step");
                e = launch_line_step(a, s);
            }
            lbm::NvtxRange r("K2 line faces");
            if (e == cudaSuccess && h->n_face_chunks > 0 && h->face_solve == 0)
                e = launch_line_faces_chunked(a, h->face_chunks, h->n_face_chunks, h->face_items, s);
            else if (e == cudaSuccess && h->n_faces > 0)
                e = launch_line_faces(a, h->faces, h->n_faces, h->face_scratch, s);
            return e;
        }
    }
    if constexpr (std::is_same<T, D>::value) {
        if (h->q == 9) {
            cudaError_t e;
            {
                lbm::NvtxRange r("K1 d2q9 step");
                e = launch_d2q9_step(a, s);
            }
            lbm::NvtxRange r("K2 d2q9 faces / edge rule");
            if (e == cudaSuccess && h->cp.macro && h->cp.mode != CRACK_NONE) e = launch_d2q9_faces(a, s);
            if (e == cudaSuccess && h->edge_macro) e = launch_edge_rule(a, s);
            return e;
        }
    }
    a.k_cta = use_k_cta(h) ? 1 : 0;
    cudaError_t e;
    {
        lbm::NvtxRange r("K1 step");
        e = launch_step(a, h->n_bands, s, h->bulk);
    }
    if (e == cudaSuccess && h->edge_macro) {
        lbm::NvtxRange r("K2 edge rule");
        e = launch_edge_rule(a, s);
    }
    return e;
}

cudaError_t enqueue_step(const lbm_handle *h, int par, cudaStream_t s)
{
    switch (h->lat.storage) {
    case LBM_F32: return enqueue_step_t<float, float>(h, par, s);
    case LBM_F32_WD_BF16: return enqueue_step_t<float, __nv_bfloat16>(h, par, s);
    case LBM_F32_WD_F16: return enqueue_step_t<float, __half>(h, par, s);
    case LBM_F32_LEAPFROG: return enqueue_step_t<float, Lf>(h, par, s);
    default: return enqueue_step_t<double, double>(h, par, s);
    }
}

const void *step_kernel_for(int storage, bool bulk = false)
{
    switch (storage) {
    case LBM_F32: return step_kernel_ptr<float, float>(bulk);
    case LBM_F32_WD_BF16: return step_kernel_ptr<float, __nv_bfloat16>(bulk);
    case LBM_F32_WD_F16: return step_kernel_ptr<float, __half>(bulk);
    case LBM_F32_LEAPFROG: return step_kernel_ptr<float, Lf>(bulk);
    default: return step_kernel_ptr<double, double>();
    }
}

// 16-bit wdot plane <-> dense FP32 array (device memory).
cudaError_t wd_to_f32(const lbm_handle *h, float *dst, double scale, cudaStream_t s)
{
    if (h->lat.storage == LBM_F32_WD_BF16)
        return launch_wd_to_f32(static_cast<const __nv_bfloat16 *>(h->wd), h->pitch, h->grid.nx, h->grid.ny, (float)scale, dst, s);
    return launch_wd_to_f32(static_cast<const __half *>(h->wd), h->pitch, h->grid.nx, h->grid.ny, (float)scale, dst, s);
}

cudaError_t wd_from_f32(const lbm_handle *h, const float *src, double scale, cudaStream_t s)
{
    if (h->lat.storage == LBM_F32_WD_BF16)
        return launch_wd_from_f32(static_cast<__nv_bfloat16 *>(h->wd), h->pitch, h->grid.nx, h->grid.ny, (float)scale, src, s);
    return launch_wd_from_f32(static_cast<__half *>(h->wd), h->pitch, h->grid.nx, h->grid.ny, (float)scale, src, s);
}

bool wd16(const lbm_handle *h) { return h->esize_d == 2; }

cudaError_t enqueue_finalize(const lbm_handle *h, cudaStream_t s)
{
    if (h->esize == 4) {
        FinalizeArgs<float> a;
        a.w = static_cast<const float *>(h->w[h->parity]);
        a.pitch = h->pitch;
        a.st = h->st + h->parity;
        a.cut_h = h->cut_h;
        a.cut_v = h->cut_v;
        a.p = h->cp;
        a.hist = h->hist;
        return h->line ? launch_line_finalize(a, s) : launch_finalize(a, s);
    }
    FinalizeArgs<double> a;
    a.w = static_cast<const double *>(h->w[h->parity]);
    a.pitch = h->pitch;
    a.st = h->st + h->parity;
    a.cut_h = h->cut_h;
    a.cut_v = h->cut_v;
    a.p = h->cp;
    a.hist = h->hist;
    return h->line ? launch_line_finalize(a, s) : launch_finalize(a, s);
}

cudaError_t drain_profile(lbm_handle *h)
{
    if (!h->ev || h->ev_used == 0) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    for (size_t q = 0; q + 2 <= h->ev_used; q += 2) {
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, (*h->ev)[q], (*h->ev)[q + 1])) != cudaSuccess) return e;
        if ((*h->ev_kind)[q / 2] == 0) { h->step_ms += ms; h->n_step += 1; }
        else { h->fin_ms += ms; h->n_fin += 1; }
    }
    h->ev_used = 0;
    return cudaSuccess;
}

// Enqueue one kernel, bracketed by events when profiling.
template <typename F>
cudaError_t timed(lbm_handle *h, int kind, F &&launch)
{
    if (!h->profiling) return launch();
    cudaError_t e;
    if (h->ev_used + 2 > h->ev->size() && (e = drain_profile(h)) != cudaSuccess) return e;
    cudaEvent_t *E = &(*h->ev)[h->ev_used];
    (*h->ev_kind)[h->ev_used / 2] = kind;
    h->ev_used += 2;
    if ((e = cudaEventRecord(E[0], h->stream)) != cudaSuccess) return e;
    if ((e = launch()) != cudaSuccess) return e;
    return cudaEventRecord(E[1], h->stream);
}

}  // namespace

namespace lbm {
namespace host {

// Apply the crack step that follows the last enqueued LBM step.
lbm_status finalize(lbm_handle *h)
{
    if (!h->pending) return LBM_OK;
    lbm::NvtxRange r("K3 crack step (finalize)");
    LBM_CUDA(timed(h, 1, [&] { return enqueue_finalize(h, h->stream); }));
    h->pending = false;
    return LBM_OK;
}

lbm_status check_sticky(lbm_handle *h)
{
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    lbm_status rc = finalize(h);
    if (rc != LBM_OK) return rc;
    CrackState hs;
    uint32_t err = 0;
    cudaError_t e = cudaMemcpyAsync(&hs, h->st + h->parity, sizeof hs, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, h->err, sizeof err, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->sticky = LBM_ERR_CUDA;
        return cuda_fail(e, "synchronising the lattice stream");
    }
    if (err & ERR_TIMEOUT) {
        h->sticky = LBM_ERR_TIMEOUT;
        return fail(LBM_ERR_TIMEOUT, "a bounded device wait gave up (grid barrier of a persistent batched step)");
    }
    if ((err & ERR_NONFINITE) || ((hs.r.flags | hs.l.flags) & FLAG_NONFINITE)) {
        h->sticky = LBM_ERR_UNSTABLE;
        return fail(LBM_ERR_UNSTABLE, "non-finite value in the fields or in K");
    }
    return LBM_OK;
}

}  // namespace host
}  // namespace lbm

namespace {

// Static partition of the rows into bands of at most `rows` rows.  The rows
// that the crack-face rule and the crack links touch form two bands of their
// own, hh rows below the crack line (ending at row jc - 1) and hh rows above
// it (starting at row jc), so that no other band holds a severed link.
std::vector<Unit> partition_rows(int ny, int rows, int jc, int hh)
{
    std::vector<Unit> v;
    auto push = [&](int j0, int j1) {
        Unit u;
        u.j0 = j0;
        u.j1 = j1;
        u.dir = 1;
        u.pad = 0;
        v.push_back(u);
    };
    auto fill = [&](int a, int b) {
        for (int j = a; j < b; j = std::min(j + rows, b)) push(j, std::min(j + rows, b));
    };
    if (hh > 0) {
        // a row slab whose boundary is the crack line holds one sub-band
        const bool below = jc >= hh, above = jc + hh <= ny;
        fill(0, below ? jc - hh : jc);
        if (below) push(jc - hh, jc);
        if (above) push(jc, jc + hh);
        fill(above ? jc + hh : jc, ny);
    } else {
        fill(0, ny);
    }
    return v;
}

// Choose the band height (rows <= 0: balance the bands over the SMs) and
// upload the unit table.
lbm_status plan_bands(lbm_handle *h, int rows)
{
    const int ny = h->grid.ny;
    const bool crack = h->cp.mode != CRACK_NONE && !h->cp.line;   // a line crack's kernel has no crack band
    const int hh = !crack ? 0 : (h->cp.macro ? 3 : 1);
    std::vector<Unit> best;
    if (rows > 0) {
        best = partition_rows(ny, rows, h->jc, hh);
    } else {
        // D2Q5: all CTAs resident at once, bands * ncb <= sms * bps, bands as
        // short as that allows; D2Q9, whose CTAs take unequal times (its
        // edge-column warps and crack rows run the general update, and it is
        // bound by instruction issue more than by memory), about three waves
        // of shorter bands, so that the dispatcher evens out the SMs' loads
        // (measured on 4096 x 2048: 5-row bands in 2.7 waves 26.7 us per
        // step, 14-row bands in one wave 28.6 us)
        const int64_t waves = h->q == 9 ? 3 : 1;
        const int64_t slots = (int64_t)h->sms * h->bps * waves;
        const int64_t nb = std::max<int64_t>(1, slots / h->ncb);
        int H = std::max(1, (int)((ny + nb - 1) / nb));
        for (;; ++H) {
            best = partition_rows(ny, H, h->jc, hh);
            if ((int64_t)best.size() * h->ncb <= slots || H >= ny) break;
        }
    }
    if ((int)best.size() > ny) return fail(LBM_ERR_ARG, "partition larger than the unit table");
    h->n_bands = (int)best.size();
    h->band_rows = 0;
    h->crack_band = -1;
    for (int b = 0; b < h->n_bands; ++b) {
        h->band_rows = std::max(h->band_rows, best[b].j1 - best[b].j0);
        // the first crack sub-band: below the crack line, else (a slab whose
        // bottom boundary is the crack line) above it
        const bool sub = h->jc >= hh ? (best[b].j0 == h->jc - hh && best[b].j1 == h->jc)
                                     : (best[b].j0 == h->jc && best[b].j1 == h->jc + hh);
        if (crack && sub && h->crack_band < 0) h->crack_band = b;
    }
    if (crack && h->crack_band < 0) return fail(LBM_ERR_ARG, "the crack rows form no band of their own");
    LBM_CUDA(cudaMemcpyAsync(h->units, best.data(), best.size() * sizeof(Unit), cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    *h->units_h = best;
    h->gen += 1;
    return LBM_OK;
}

void *dev_alloc(lbm_handle *h, size_t bytes)
{
    if (h->custom_alloc) return h->alloc.alloc(bytes, h->alloc.ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    return p;
}

void dev_free(lbm_handle *h, void *p)
{
    if (!p) return;
    if (h->custom_alloc) h->alloc.release(p, h->alloc.ctx);
    else cudaFree(p);
}

void free_host(lbm_handle *h)
{
    delete h->units_h;
    delete h->init_cut;
    delete h;
}

void drop_graph(lbm_handle *h) { h->steps.reset(); }

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                      const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads,
                      void *stream, const lbm_allocator *allocator, lbm_handle **out)
{
    return create_impl(grid, lattice, material, crack, loads, n_loads, stream, allocator, false, out);
}

lbm_status lbm_create_line(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                           const lbm_crack_line *crack, const lbm_loading *loads, int32_t n_loads,
                           void *stream, const lbm_allocator *allocator, lbm_handle **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !lattice || !material || !crack) return fail(LBM_ERR_ARG, "grid, lattice, material and crack are required");
    const lbm_crack_line &c = *crack;
    if (c.mode < LBM_CRACK_STATIONARY || c.mode > LBM_CRACK_KCRIT)
        return fail(LBM_ERR_ARG, "a crack in any direction needs a stationary, prescribed or K-criterion mode");
    if (lattice->velocity_set != LBM_D2Q5) return fail(LBM_ERR_ARG, "a crack in any direction is built for D2Q5");
    if (lattice->bc_mode != LBM_BC_BOUNCEBACK && lattice->bc_mode != LBM_BC_MACROSCOPIC)
        return fail(LBM_ERR_ARG, "a crack in any direction is built with link-local edges (LBM_BC_BOUNCEBACK or LBM_BC_MACROSCOPIC)");
    if (lattice->storage < LBM_F64 || lattice->storage > LBM_F32_WD_F16) return fail(LBM_ERR_ARG, "unknown storage");
    if (grid->nx < 1 || grid->ny < 2 || !(grid->dh > 0.0) || !std::isfinite(grid->dh))
        return fail(LBM_ERR_ARG, "need nx >= 1, ny >= 2 and a positive, finite dh");
    if (c.mode == LBM_CRACK_PRESCRIBED && !(c.v_rel >= 0.0 && c.v_rel < 1.0))
        return fail(LBM_ERR_ARG, "prescribed v_rel must lie in [0, 1)");
    if (c.mode == LBM_CRACK_KCRIT && !(c.K_C > 0.0 && c.v_max >= 0.0 && c.v_max < 1.0))
        return fail(LBM_ERR_ARG, "K-criterion needs K_C > 0 and 0 <= v_max < 1");
    const double rmin = c.r_min > 0.0 ? c.r_min : c.r0;
    if (!(rmin > 0.5 * grid->dh))
        return fail(LBM_ERR_ARG, "the K window must start more than dh / 2 behind the tip (r0 or r_min)");
    const double pts[4] = {c.x_start / grid->dh, c.y_start / grid->dh, c.x_tip / grid->dh, c.y_tip / grid->dh};
    const double lim[4] = {(double)grid->nx, (double)grid->ny, (double)grid->nx, (double)grid->ny};
    for (int q = 0; q < 4; ++q)
        if (!(pts[q] >= 0.0 && pts[q] <= lim[q])) return fail(LBM_ERR_ARG, "the crack's start and tip must lie in the body");
    LineSpec L;
    L.start_xq = llrint(c.x_start / grid->dh * 4294967296.0);
    L.start_yq = llrint(c.y_start / grid->dh * 4294967296.0);
    L.tip_xq = llrint(c.x_tip / grid->dh * 4294967296.0);
    L.tip_yq = llrint(c.y_tip / grid->dh * 4294967296.0);
    const int64_t X = (int64_t)grid->nx << kQBits, Y = (int64_t)grid->ny << kQBits;
    if (L.start_xq < 0 || L.start_xq > X || L.tip_xq < 0 || L.tip_xq > X || L.start_yq < 0 || L.start_yq > Y ||
        L.tip_yq < 0 || L.tip_yq > Y)
        return fail(LBM_ERR_ARG, "the crack's start and tip must lie in the body");
    if (L.start_xq == L.tip_xq && L.start_yq == L.tip_yq) return fail(LBM_ERR_ARG, "the crack's start and tip coincide");
    // the unit direction, its products kept apart from the sum (no fused
    // multiply-add), as every implementation of this reading forms it
    volatile double dx = (double)(L.tip_xq - L.start_xq), dy = (double)(L.tip_yq - L.start_yq);
    volatile double xx = dx * dx, yy = dy * dy;
    const double len = std::sqrt(xx + yy);
    L.dir_x = dx / len;
    L.dir_y = dy / len;
    if (line_hits_a_centre(L, grid->nx, grid->ny)) return fail(LBM_ERR_ARG, "the crack's line passes through a site centre");
    if (lattice->bc_mode == LBM_BC_MACROSCOPIC) {
        // every point of the initial crack (a site with a severed link) needs
        // its x_I and x_II cells inside the body
        std::vector<uint8_t> dropped;
        const std::vector<LineFace> tab = line_faces_table(L, grid->nx, grid->ny, &dropped);
        const int words = (grid->nx + 31) / 32;
        const std::vector<uint32_t> m = line_initial_masks(L, grid->nx, grid->ny, words);
        const size_t vo = (size_t)grid->ny * words;
        auto cut = [&](size_t off, int i, int j) { return ((m[off + (size_t)j * words + (size_t)(i >> 5)] >> (i & 31)) & 1u) != 0; };
        for (size_t q = 0; q < tab.size(); ++q) {
            if (!dropped[q]) continue;
            const int i = tab[q].i, j = tab[q].j;
            if (cut(0, i, j) || (i >= 1 && cut(0, i - 1, j)) || (j + 1 < grid->ny && cut(vo, i, j)) || (j >= 1 && cut(vo, i, j - 1)))
                return fail(LBM_ERR_ARG, "macroscopic crack faces: a point of the initial crack has its x_I or x_II cell outside the body (keep the crack two spacings from the edges)");
        }
    }
    // the rows its links can touch: from the start to where the line leaves
    // the body, widened by three rows
    const double sx = (double)L.start_xq * kTwoM32, sy = (double)L.start_yq * kTwoM32;
    const double tx = L.dir_x > 0.0 ? ((double)grid->nx - sx) / L.dir_x : (L.dir_x < 0.0 ? -sx / L.dir_x : 1e300);
    const double ty = L.dir_y > 0.0 ? ((double)grid->ny - sy) / L.dir_y : (L.dir_y < 0.0 ? -sy / L.dir_y : 1e300);
    const double ey = sy + std::min(tx, ty) * L.dir_y;
    L.row_lo = (int32_t)std::max(0.0, std::floor(std::min(sy, ey)) - 3.0);
    L.row_hi = (int32_t)std::min((double)grid->ny - 1.0, std::floor(std::max(sy, ey)) + 3.0);
    if (c.two_tips != 0 && c.two_tips != 1) return fail(LBM_ERR_ARG, "two_tips must be 0 or 1");
    lbm_crack cr;
    std::memset(&cr, 0, sizeof cr);
    cr.mode = c.mode;
    cr.two_tips = c.two_tips;
    cr.x_start = c.x_start;
    cr.x_tip = c.x_tip;
    cr.v_rel = c.v_rel;
    cr.K_C = c.K_C;
    cr.v_max = c.v_max;
    cr.r0 = c.r0;
    cr.r_min = c.r_min;
    cr.fit_width = c.fit_width;
    cr.hist_cap = c.hist_cap;
    return create_impl(grid, lattice, material, &cr, loads, n_loads, stream, allocator, false, out, &L);
}

}  // extern "C"

namespace lbm {
namespace host {

// The scale of FP16 wdot storage (stored = wdot * scale): a power of two
// that puts the largest rate the Dirichlet loads impose near 2^10, leaving a
// factor 64 below FP16's largest value for waves.
double fp16_wd_scale(const lbm_grid *grid, const lbm_loading *loads, int32_t n_loads)
{
    double rate = 0.0;
    for (int r = 0; r < n_loads; ++r) {
        const lbm_loading &L = loads[r];
        if (L.edge < 0 || L.edge > 3 || grid->edge[L.edge] != LBM_EDGE_DIRICHLET) continue;
        const double T = L.t_ramp > grid->dt ? L.t_ramp : grid->dt;
        if (L.kind == LBM_LOAD_LINEAR) rate = std::max(rate, std::fabs(L.amp) / T);
        else if (L.kind == LBM_LOAD_SIN2 || L.kind == LBM_LOAD_HALFSINE) rate = std::max(rate, 3.2 * std::fabs(L.amp) / T);
        else if (L.kind == LBM_LOAD_SERIES)
            for (int64_t k = 1; L.series && k < L.n_series; ++k)
                rate = std::max(rate, std::fabs(L.series[k] - L.series[k - 1]) / grid->dt);
    }
    double scale = rate > 0.0 ? std::ldexp(1.0, 10 - (int)std::ceil(std::log2(rate))) : 1024.0;
    return std::min(std::max(scale, std::ldexp(1.0, -40)), std::ldexp(1.0, 60));
}

lbm_status create_impl(const lbm_grid *grid, const lbm_lattice *lattice, const lbm_material *material,
                       const lbm_crack *crack, const lbm_loading *loads, int32_t n_loads, void *stream,
                       const lbm_allocator *allocator, bool slab, lbm_handle **out, const LineSpec *line)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !lattice || !material) return fail(LBM_ERR_ARG, "grid, lattice and material are required");
    if (grid->nx < 1 || grid->ny < 2) return fail(LBM_ERR_ARG, "need nx >= 1 and ny >= 2");
    if ((int64_t)grid->nx * grid->ny > ((int64_t)1 << 34)) return fail(LBM_ERR_ARG, "lattice too large");
    if (!(grid->dh > 0.0) || !(grid->dt > 0.0) || !std::isfinite(grid->dh) || !std::isfinite(grid->dt))
        return fail(LBM_ERR_ARG, "dh and dt must be positive and finite");
    for (int e = 0; e < 4; ++e)
        if (grid->edge[e] < LBM_EDGE_FREE ||
            grid->edge[e] > (slab && (e == LBM_BOTTOM || e == LBM_TOP) ? (int)EDGE_HALO : LBM_EDGE_PERIODIC))
            return fail(LBM_ERR_ARG, "unknown edge kind");
    if ((grid->edge[LBM_LEFT] == LBM_EDGE_PERIODIC) != (grid->edge[LBM_RIGHT] == LBM_EDGE_PERIODIC) ||
        (grid->edge[LBM_BOTTOM] == LBM_EDGE_PERIODIC) != (grid->edge[LBM_TOP] == LBM_EDGE_PERIODIC))
        return fail(LBM_ERR_ARG, "periodic edges must come in opposite pairs");
    if (lattice->velocity_set != LBM_D2Q5 && lattice->velocity_set != LBM_D2Q9)
        return fail(LBM_ERR_ARG, "unknown velocity set (D2Q5 or D2Q9)");
    const bool d2q9 = lattice->velocity_set == LBM_D2Q9;
    if (d2q9 && lattice->storage != LBM_F64 && lattice->storage != LBM_F32)
        return fail(LBM_ERR_ARG, "D2Q9 needs LBM_F64 or LBM_F32 storage");
    if (lattice->form != LBM_FORM_MOMENT) return fail(LBM_ERR_ARG, "only the moment form is built");
    if (lattice->omega != 1.0) return fail(LBM_ERR_ARG, "omega = dt/tau must be 1 (tau = dt)");
    if (lattice->storage < LBM_F64 || lattice->storage > LBM_F32_LEAPFROG) return fail(LBM_ERR_ARG, "unknown storage");
    if (lattice->bc_mode < LBM_BC_BOUNCEBACK || lattice->bc_mode > LBM_BC_MACROSCOPIC_EDGES)
        return fail(LBM_ERR_ARG, "unknown boundary mode");
    const bool macro_faces = lattice->bc_mode != LBM_BC_BOUNCEBACK;
    const bool macro_edges = lattice->bc_mode == LBM_BC_MACROSCOPIC_EDGES;
    if (macro_edges) {
        // x_II of an edge point must not be a boundary point of the opposite
        // edge; in a row slab, x_II of a point of a ruled bottom or top edge,
        // and the edge points a corner reads, must lie in the slab (its halo
        // rows hold the previous step's rows when the rule runs): a slab
        // takes at least four rows
        if (grid->edge[LBM_LEFT] != LBM_EDGE_PERIODIC && grid->nx < 4)
            return fail(LBM_ERR_ARG, "the macroscopic edge rule needs nx >= 4 between free or Dirichlet edges");
        if (grid->edge[LBM_BOTTOM] != LBM_EDGE_PERIODIC && grid->ny < 4)
            return fail(LBM_ERR_ARG, "the macroscopic edge rule needs ny >= 4 between free or Dirichlet edges");
    }
    if (!(material->rho > 0.0) || !(material->mu > 0.0) || !std::isfinite(material->rho) || !std::isfinite(material->mu))
        return fail(LBM_ERR_ARG, "rho and mu must be positive and finite");
    const double cs = std::sqrt(material->mu / material->rho);
    const double g = cs * cs * grid->dt / (grid->dh * grid->dh);
    if (g * grid->dt > (d2q9 ? 0.75 : 0.5))
        return fail(LBM_ERR_ARG, d2q9 ? "unstable: c_s^2 dt^2 / dh^2 > 3/4" : "unstable: c_s^2 dt^2 / dh^2 > 1/2");

    lbm_crack cr;
    std::memset(&cr, 0, sizeof cr);
    if (crack) cr = *crack;
    if (cr.mode < LBM_CRACK_NONE || cr.mode > LBM_CRACK_KCRIT) return fail(LBM_ERR_ARG, "unknown crack mode");
    int32_t jc = 0;
    int64_t start_q = 0, tip_q = 0;
    const int64_t qone = (int64_t)1 << kQBits;
    const int64_t clamp_q = (int64_t)grid->nx * qone;   // the far edge: the crack splits the body
    if (line) {
        // a crack in any direction, validated by lbm_create_line
        start_q = line->start_xq;
        tip_q = line->tip_xq;
        if (!(cr.fit_width > 0.0)) cr.fit_width = grid->dh;
        if (cr.hist_cap <= 0) cr.hist_cap = kDefaultHistCap;
    } else if (cr.mode != LBM_CRACK_NONE) {
        const double yj = cr.y / grid->dh;
        if (!std::isfinite(yj) || std::fabs(yj - std::nearbyint(yj)) > 1e-9)
            return fail(LBM_ERR_ARG, "the crack line y must be a multiple of dh (between two rows)");
        jc = (int32_t)std::nearbyint(yj);
        // the crack rows keep `margin` rows from a bottom or top edge; from a
        // row slab's halo edge they need only lie inside the slab
        const int margin = macro_edges ? 4 : (macro_faces ? 3 : 1);
        const int margin_lo = grid->edge[LBM_BOTTOM] == EDGE_HALO ? (macro_faces ? 3 : 1) : margin;
        const int margin_hi = grid->edge[LBM_TOP] == EDGE_HALO ? (macro_faces ? 3 : 1) : margin;
        // a row slab may have the crack line on a halo boundary (the
        // neighbouring slab holds the other side's rows)
        const bool on_lo = slab && jc == 0 && grid->edge[LBM_BOTTOM] == EDGE_HALO;
        const bool on_hi = slab && jc == grid->ny && grid->edge[LBM_TOP] == EDGE_HALO;
        const int hh_rows = macro_faces ? 3 : 1;
        // a D2Q9 slab holds both sides' crack rows: its crack step, diagonal
        // cuts and face rule read the rows on both sides of the line
        if (d2q9 && (on_lo || on_hi))
            return fail(LBM_ERR_ARG, "a D2Q9 row slab needs the crack rows of both sides of the crack line inside it");
        if (on_lo || on_hi) {
            if (grid->ny < hh_rows + (on_lo && on_hi ? hh_rows : 0))
                return fail(LBM_ERR_ARG, "a slab whose boundary is the crack line needs the crack rows of its side");
        } else if (jc < margin_lo || jc > grid->ny - margin_hi) {
            return fail(LBM_ERR_ARG, "the crack line is too close to the bottom or top edge");
        }
        if (!(cr.x_start >= 0.0) || !(cr.x_tip >= cr.x_start)) return fail(LBM_ERR_ARG, "need 0 <= x_start <= x_tip");
        start_q = llrint(cr.x_start / grid->dh * 4294967296.0);
        tip_q = llrint(cr.x_tip / grid->dh * 4294967296.0);
        if (tip_q >= clamp_q) return fail(LBM_ERR_ARG, "the initial tip must lie left of x = nx dh");
        if (macro_faces && grid->edge[LBM_LEFT] == LBM_EDGE_PERIODIC)
            return fail(LBM_ERR_ARG, "macroscopic crack faces need non-periodic left/right edges");
        if (cr.mode == LBM_CRACK_PRESCRIBED && !(cr.v_rel >= 0.0 && cr.v_rel < 1.0))
            return fail(LBM_ERR_ARG, "prescribed v_rel must lie in [0, 1)");
        if (cr.two_tips != 0 && cr.two_tips != 1) return fail(LBM_ERR_ARG, "two_tips must be 0 or 1");
        if (cr.mode == LBM_CRACK_KCRIT && !(cr.K_C > 0.0 && cr.v_max >= 0.0 && cr.v_max < 1.0))
            return fail(LBM_ERR_ARG, "K-criterion needs K_C > 0 and 0 <= v_max < 1");
        if (!(cr.r_min > 0.0) && !(cr.r0 >= 0.0)) return fail(LBM_ERR_ARG, "r0 must be >= 0");
        if (macro_faces) {
            // With the macroscopic crack-face rule a narrow intact ligament between
            // a crack end and an edge carries a mode that grows without bound: one
            // column at a link-local free edge, two columns at a link-local
            // Dirichlet edge or at any edge under the macroscopic edge rule.  None,
            // or five columns and more, are fine.
            const int64_t half = qone / 2;
            const int64_t first = -floor_div(-(start_q - half), qone), last = floor_div(tip_q - half, qone);
            auto unstable = [&](int64_t width, int32_t kind) {
                if (kind == LBM_EDGE_PERIODIC) return false;
                if (macro_edges) return width == 2;
                return width == (kind == LBM_EDGE_FREE ? 1 : 2);
            };
            if (last >= first && (unstable(first, grid->edge[LBM_LEFT]) ||
                                  unstable(grid->nx - 1 - last, grid->edge[LBM_RIGHT])))
                return fail(LBM_ERR_ARG, "macroscopic crack faces: the crack leaves an unstable narrow ligament at an edge");
        }
        if (!(cr.fit_width > 0.0)) cr.fit_width = grid->dh;
        if (cr.hist_cap <= 0) cr.hist_cap = kDefaultHistCap;
    }
    if (n_loads < 0 || (n_loads > 0 && !loads)) return fail(LBM_ERR_ARG, "bad loads array");

    lbm_handle *h = new (std::nothrow) lbm_handle;
    if (!h) return fail(LBM_ERR_OOM, "host allocation failed");
    std::memset(h, 0, sizeof *h);
    h->grid = *grid;
    // the kernels of consecutive steps chained by programmatic dependent
    // launch on small lattices, whose steps are bound by launch latency
    // (measured: 98 K sites 5 % faster chained, 1 M sites 9 % slower)
    h->chained = (int64_t)grid->nx * grid->ny <= kChainedSites;
    h->lat = *lattice;
    h->mat = *material;
    h->crack = cr;
    h->jc = jc;
    h->esize = lattice->storage == LBM_F64 ? 8 : 4;
    // leapfrog storage has no wdot plane (its "wdot plane" is the other w buffer)
    h->esize_d = lattice->storage == LBM_F64 ? 8
               : lattice->storage == LBM_F32 ? 4
               : lattice->storage == LBM_F32_LEAPFROG ? 0 : 2;
    h->g = g;
    h->stream = (cudaStream_t)stream;
    h->sticky = LBM_OK;
    h->steps.gen = -1;
    h->units_h = new (std::nothrow) std::vector<Unit>();
    h->init_cut = new (std::nothrow) std::vector<uint32_t>();
    if (!h->units_h || !h->init_cut) {
        delete h->units_h;
        delete h->init_cut;
        delete h;
        return fail(LBM_ERR_OOM, "host allocation failed");
    }
    if (allocator && allocator->alloc && allocator->release) {
        h->alloc = *allocator;
        h->custom_alloc = true;
    }
    std::vector<int> seen(4, 0);
    for (int q = 0; q < n_loads; ++q) {
        const lbm_loading &L = loads[q];
        if (L.edge < 0 || L.edge > 3 || seen[L.edge]) { free_host(h); return fail(LBM_ERR_ARG, "bad or repeated load edge"); }
        if (L.kind < LBM_LOAD_ZERO || L.kind > LBM_LOAD_CONST) { free_host(h); return fail(LBM_ERR_ARG, "unknown load kind"); }
        if (L.kind == LBM_LOAD_SERIES && (!L.series || L.n_series <= 0)) { free_host(h); return fail(LBM_ERR_ARG, "series load without data"); }
        seen[L.edge] = 1;
        h->load[L.edge].kind = L.kind;
        h->load[L.edge].amp = L.amp;
        h->load[L.edge].t = L.t_ramp;
        h->load[L.edge].n = L.kind == LBM_LOAD_SERIES ? L.n_series : 0;
        h->series_cap[L.edge] = h->load[L.edge].n;
    }

    // step kernel shape: a thread per 16-byte vector of a row, kThreads a CTA
    const int vec = (int)(16 / h->esize);
    const int cols = kThreads * vec;
    h->ncb = (grid->nx + cols - 1) / cols;
    const void *kfn = step_kernel_for(lattice->storage);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->bps, kfn, kThreads, 0);
    if (e != cudaSuccess) { free_host(h); return cuda_fail(e, "querying the device"); }
    if (h->bps < 1) { free_host(h); return fail(LBM_ERR_ARG, "the step kernel does not fit on an SM"); }

    const int64_t xoff = 128 / (int64_t)h->esize;
    h->pitch = xoff + (int64_t)h->ncb * cols + xoff;
    h->words = (grid->nx + 31) / 32;
    const int64_t hcap = cr.mode != LBM_CRACK_NONE ? cr.hist_cap : 1;

    // one block for everything, carved at 256-byte boundaries
    const size_t plane = (size_t)(grid->ny + 2) * (size_t)h->pitch * h->esize;
    const size_t plane_d = (size_t)(grid->ny + 2) * (size_t)h->pitch * h->esize_d;
    const size_t staging = (h->esize_d == 2 || h->esize_d == 0) ? (size_t)grid->nx * grid->ny * 4 : 0;
    const size_t mask = (size_t)grid->ny * (size_t)h->words * 4;
    // the V mask has one more row below row 0: the links across the bottom
    // boundary of a row slab whose boundary is the crack line
    const size_t mask_v = mask + (size_t)h->words * 4;
    size_t off = 0;
    const size_t o_w0 = off; off = align256(off + plane);
    const size_t o_w1 = off; off = align256(off + plane);
    const size_t o_wd = off; off = align256(off + plane_d);
    const size_t o_sg = off; off = align256(off + staging);
    const size_t o_ch = off; off = align256(off + mask);
    const size_t o_cv = off; off = align256(off + mask_v);
    const size_t o_st = off; off = align256(off + 2 * sizeof(CrackState));
    const size_t o_er = off; off = align256(off + sizeof(uint32_t));
    const size_t o_un = off; off = align256(off + (size_t)grid->ny * sizeof(Unit));
    const size_t o_hK = off; off = align256(off + (size_t)hcap * 8);
    const size_t o_hv = off; off = align256(off + (size_t)hcap * 8);
    const size_t o_ht = off; off = align256(off + (size_t)hcap * 8);
    const size_t o_hn = off; off = align256(off + (size_t)hcap * 4);
    if (cr.mode == LBM_CRACK_NONE) cr.two_tips = 0;
    const int64_t hcap_l = cr.two_tips ? hcap : 1;   // records of the left end
    const size_t o_hKl = off; off = align256(off + (size_t)hcap_l * 8);
    const size_t o_hvl = off; off = align256(off + (size_t)hcap_l * 8);
    const size_t o_htl = off; off = align256(off + (size_t)hcap_l * 8);
    const size_t o_hnl = off; off = align256(off + (size_t)hcap_l * 4);
    // the tips' y of a crack in any direction
    const size_t o_hty = off; off = align256(off + (size_t)(line ? hcap : 1) * 8);
    const size_t o_htyl = off; off = align256(off + (size_t)(line ? hcap_l : 1) * 8);
    size_t o_ser[4];
    for (int q = 0; q < 4; ++q) { o_ser[q] = off; off = align256(off + (size_t)h->load[q].n * 8); }
    h->block_bytes = off;
    h->block = dev_alloc(h, off);
    if (!h->block) { free_host(h); return fail(LBM_ERR_OOM, "device allocation failed"); }
    char *base = static_cast<char *>(h->block);
    const size_t origin = ((size_t)h->pitch + (size_t)xoff) * h->esize;   // row 0, column 0
    h->w[0] = base + o_w0 + origin;
    h->w[1] = base + o_w1 + origin;
    h->wd = h->esize_d ? base + o_wd + ((size_t)h->pitch + (size_t)xoff) * h->esize_d : nullptr;
    h->wbase[0] = base + o_w0;
    h->wbase[1] = base + o_w1;
    h->wdbase = base + o_wd;
    h->plane_bytes = plane;
    h->plane_d_bytes = plane_d;
    h->staging = staging ? reinterpret_cast<float *>(base + o_sg) : nullptr;
    h->cut_h = reinterpret_cast<uint32_t *>(base + o_ch);
    h->cut_v = reinterpret_cast<uint32_t *>(base + o_cv) + h->words;
    h->st = reinterpret_cast<CrackState *>(base + o_st);
    h->err = reinterpret_cast<uint32_t *>(base + o_er);
    h->units = reinterpret_cast<Unit *>(base + o_un);
    h->hist.K = reinterpret_cast<double *>(base + o_hK);
    h->hist.v = reinterpret_cast<double *>(base + o_hv);
    h->hist.tip = reinterpret_cast<int64_t *>(base + o_ht);
    h->hist.np = reinterpret_cast<int32_t *>(base + o_hn);
    h->hist.Kl = reinterpret_cast<double *>(base + o_hKl);
    h->hist.vl = reinterpret_cast<double *>(base + o_hvl);
    h->hist.tipl = reinterpret_cast<int64_t *>(base + o_htl);
    h->hist.npl = reinterpret_cast<int32_t *>(base + o_hnl);
    h->hist.tipy = reinterpret_cast<int64_t *>(base + o_hty);
    h->hist.tipyl = reinterpret_cast<int64_t *>(base + o_htyl);

    cudaStream_t s = h->stream;
    auto bail = [&](lbm_status rc) {
        cudaStreamSynchronize(s);
        dev_free(h, h->block);
        free_host(h);
        return rc;
    };
    e = cudaMemsetAsync(h->block, 0, h->block_bytes, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "clearing device state"));
    for (int q = 0; q < 4; ++q) {
        if (h->load[q].kind != LBM_LOAD_SERIES) continue;
        const lbm_loading *L = nullptr;
        for (int r = 0; r < n_loads; ++r) if (loads[r].edge == q) L = &loads[r];
        double *dser = reinterpret_cast<double *>(base + o_ser[q]);
        e = cudaMemcpyAsync(dser, L->series, (size_t)L->n_series * 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "copying a load series"));
        h->load[q].series = dser;
    }
    e = cudaStreamSynchronize(s);   // the caller's series buffers may go away after create
    if (e != cudaSuccess) return bail(cuda_fail(e, "copying load series"));

    CrackParams &cp = h->cp;
    std::memset(&cp, 0, sizeof cp);
    cp.mode = cr.mode;
    cp.jc = jc;
    cp.nx = grid->nx;
    cp.ny = grid->ny;
    cp.macro = macro_faces;
    {
        const int hh_rows = macro_faces ? 3 : 1;
        cp.sides = (jc >= hh_rows ? 1 : 0) | (jc + hh_rows <= grid->ny ? 2 : 0);
    }
    h->edge_macro = macro_edges;
    h->q = d2q9 ? 9 : 5;
    cp.words = h->words;
    cp.two_tips = cr.two_tips ? 1 : 0;
    cp.q = d2q9 ? 9 : 5;
    cp.mu = material->mu;
    cp.cs = cs;
    cp.dt = grid->dt;
    cp.dh = grid->dh;
    cp.K_C = cr.K_C;
    cp.v_max = cr.v_max;
    cp.r0 = cr.r0;
    cp.r_min_fixed = cr.r_min;
    cp.fit_width = cr.fit_width;
    cp.v_rel = cr.v_rel;
    cp.start_q = start_q;
    cp.clamp_q = clamp_q;
    h->line = line != nullptr;
    if (line) {
        cp.line = 1;
        cp.dir_x = line->dir_x;
        cp.dir_y = line->dir_y;
        cp.row_lo = line->row_lo;
        cp.row_hi = line->row_hi;
        cp.clamp_yq = (int64_t)grid->ny * qone;
        cp.start_yq = line->start_yq;
        // bands as short as keeps every CTA of the step resident at once
        int bps_line = 0;
        const void *lk = lattice->storage == LBM_F64           ? line_step_kernel_ptr<double, double>()
                         : lattice->storage == LBM_F32_WD_BF16 ? line_step_kernel_ptr<float, __nv_bfloat16>()
                         : lattice->storage == LBM_F32_WD_F16  ? line_step_kernel_ptr<float, __half>()
                                                               : line_step_kernel_ptr<float, float>();
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_line, lk, kThreads, 0);
        if (e != cudaSuccess) return bail(cuda_fail(e, "querying the line step kernel"));
        // every slot but the tip block's goes to the march
        const int64_t slots = (int64_t)h->sms * std::max(bps_line, 1) - 1;
        const int64_t nb = std::max<int64_t>(1, slots / h->ncb);
        cp.band = (int32_t)std::max<int64_t>(1, (grid->ny + nb - 1) / nb);
        h->line_band0 = cp.band;
        if (macro_faces) {
            // the macroscopic rule on the crack's faces: the tabulated points
            const std::vector<LineFace> tab = line_faces_table(*line, grid->nx, grid->ny);
            h->n_faces = (int32_t)tab.size();
            std::vector<lbm::FaceChunk> chunks;
            std::vector<lbm::FaceItem> items;
            const bool chunked = !tab.empty() && line_face_chunks(tab, chunks, items);
            if (!tab.empty()) {
                // the table, the chunk tables (the chunked solve, where the
                // coupling allows it) and the one-CTA solve's scratch
                const size_t o_ch = align256(tab.size() * sizeof(LineFace));
                const size_t o_it = o_ch + align256(chunks.size() * sizeof(lbm::FaceChunk));
                const size_t fbytes = o_it + items.size() * sizeof(lbm::FaceItem);
                h->faces = static_cast<LineFace *>(dev_alloc(h, fbytes));
                h->face_scratch = static_cast<double *>(dev_alloc(h, tab.size() * lbm::kLineFaceScratch));
                if (!h->faces || !h->face_scratch) {
                    dev_free(h, h->faces);
                    dev_free(h, h->face_scratch);
                    return bail(fail(LBM_ERR_OOM, "device allocation failed"));
                }
                e = cudaMemcpyAsync(h->faces, tab.data(), tab.size() * sizeof(LineFace), cudaMemcpyHostToDevice, s);
                if (chunked) {
                    char *base = reinterpret_cast<char *>(h->faces);
                    h->face_chunks = reinterpret_cast<lbm::FaceChunk *>(base + o_ch);
                    h->face_items = reinterpret_cast<lbm::FaceItem *>(base + o_it);
                    h->n_face_chunks = (int32_t)chunks.size();
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(h->face_chunks, chunks.data(), chunks.size() * sizeof(lbm::FaceChunk),
                                            cudaMemcpyHostToDevice, s);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(h->face_items, items.data(), items.size() * sizeof(lbm::FaceItem),
                                            cudaMemcpyHostToDevice, s);
                }
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) {
                    dev_free(h, h->faces);
                    dev_free(h, h->face_scratch);
                    return bail(cuda_fail(e, "writing the boundary points"));
                }
            }
        }
    }
    cp.hist_cap = cr.mode != LBM_CRACK_NONE ? cr.hist_cap : 0;
    // ((v c_s) dt / dh) 2^32, rounded to nearest (even): the crack step's own
    // expression for the advance, formed once
    cp.dq_prescribed = cr.mode == LBM_CRACK_PRESCRIBED ? llrint(cr.v_rel * cs * grid->dt / grid->dh * 4294967296.0) : 0;
    cp.dq_max = cr.mode == LBM_CRACK_KCRIT ? llrint(cr.v_max * cs * grid->dt / grid->dh * 4294967296.0) + 1 : 0;

    h->wd_scale = lattice->storage == LBM_F32_WD_F16 ? fp16_wd_scale(grid, loads, n_loads) : 1.0;

    lbm_status rc = plan_bands(h, 0);
    if (rc != LBM_OK) return bail(rc);

    // initial state: the initial crack's links (x_start <= x_i <= x_tip) severed
    CrackState hs;
    std::memset(&hs, 0, sizeof hs);
    hs.r.tip_q = tip_q;
    hs.l.tip_q = start_q;
    hs.i_first = 0;
    hs.i_last = -1;
    hs.r.decided = 1;
    hs.l.decided = 1;
    std::vector<uint32_t> row((size_t)h->words, 0u);
    if (line) {
        // every H and V link the initial segment meets, in exact arithmetic;
        // kept as [H mask | V mask] for lbm_reset
        hs.r.tip_q = line->tip_xq;
        hs.r.tip_yq = line->tip_yq;
        hs.l.tip_q = line->start_xq;
        hs.l.tip_yq = line->start_yq;
        hs.r.v_prev = cr.mode == LBM_CRACK_PRESCRIBED ? cr.v_rel : 0.0;
        hs.l.v_prev = hs.r.v_prev;
        row = line_initial_masks(*line, grid->nx, grid->ny, h->words);
        const size_t n = (size_t)grid->ny * h->words;
        e = cudaMemcpyAsync(h->cut_h, row.data(), n * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->cut_v, row.data() + n, n * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "writing the initial crack"));
    } else if (cr.mode != LBM_CRACK_NONE) {
        const int64_t half = qone / 2;
        int64_t first = -floor_div(-(start_q - half), qone);   // smallest i with x_i >= x_start
        int64_t last = floor_div(tip_q - half, qone);          // largest i with x_i <= x_tip
        if (first < 0) first = 0;
        if (last > grid->nx - 1) last = grid->nx - 1;
        hs.i_first = (int32_t)first;
        hs.i_last = (int32_t)(last < first ? first - 1 : last);
        hs.r.v_prev = cr.mode == LBM_CRACK_PRESCRIBED ? cr.v_rel : 0.0;
        hs.l.v_prev = hs.r.v_prev;
        for (int i = hs.i_first; i <= hs.i_last; ++i) row[(size_t)(i >> 5)] |= 1u << (i & 31);
        e = cudaMemcpyAsync(h->cut_v + (ptrdiff_t)(jc - 1) * h->words, row.data(), row.size() * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "writing the initial crack"));
    }
    h->init_st = hs;
    *h->init_cut = row;
    e = cudaMemcpyAsync(h->st, &hs, sizeof hs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_wstar(h->st, h->load, h->grid.edge, grid->dt, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors go out of scope
    if (e != cudaSuccess) return bail(cuda_fail(e, "initialising the crack state"));
    e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "creating the capture stream"));
    *out = h;
    clear_error();
    return LBM_OK;
}

}  // namespace host
}  // namespace lbm

extern "C" {

lbm_status lbm_step(lbm_handle *h, int64_t n)
{
    lbm::NvtxRange nvtx_("lbm_step");
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
    if (n > 0 && h->cp.mode != CRACK_NONE) h->pending = true;
    if (!h->profiling) {
        // runs of steps replay graphs of 64, 32, ..., 2 steps
        int par = h->parity;
        const lbm_status rc = run_chunks(h->steps, h->gen, h->stream, h->cap_stream, n, par,
                                         [&](int p, cudaStream_t s) { return enqueue_step(h, p, s); });
        h->parity = par;
        return rc;
    }
    while (n > 0) {
        LBM_CUDA(timed(h, 0, [&] { return enqueue_step(h, h->parity, h->stream); }));
        h->parity ^= 1;
        n -= 1;
    }
    return LBM_OK;
}

// The dtype a field is exchanged in: the arithmetic precision (FP64 for F64
// storage, FP32 otherwise; 16-bit wdot planes are converted).
static int32_t exchange_dtype(const lbm_handle *h) { return h->esize == 8 ? LBM_F64 : LBM_F32; }

lbm_status lbm_fields(lbm_handle *h, int32_t which, void *dst, int32_t dst_on_device, int32_t dtype)
{
    lbm::NvtxRange nvtx_("lbm_fields");
    if (!h || !dst) return fail(LBM_ERR_ARG, "handle or dst is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (which != LBM_FIELD_W && which != LBM_FIELD_WDOT) return fail(LBM_ERR_ARG, "unknown field");
    if (dtype != exchange_dtype(h)) return fail(LBM_ERR_ARG, "dtype must be LBM_F64 for F64 storage, LBM_F32 otherwise");
    const size_t row = (size_t)h->grid.nx * h->esize;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (which == LBM_FIELD_WDOT && h->esize_d == 0) {
        // leapfrog storage: wdot_n = (w_n - w_{n-1}) / dt
        float *conv = dst_on_device ? static_cast<float *>(dst) : h->staging;
        LBM_CUDA(launch_lf_wdot(static_cast<const float *>(h->w[h->parity]), static_cast<const float *>(h->w[h->parity ^ 1]),
                                h->pitch, h->grid.nx, h->grid.ny, (float)h->grid.dt, conv, h->stream));
        if (!dst_on_device)
            LBM_CUDA(cudaMemcpyAsync(dst, conv, (size_t)h->grid.nx * h->grid.ny * 4, cudaMemcpyDeviceToHost, h->stream));
    } else if (which == LBM_FIELD_WDOT && wd16(h)) {
        float *conv = dst_on_device ? static_cast<float *>(dst) : h->staging;
        LBM_CUDA(wd_to_f32(h, conv, h->wd_scale, h->stream));
        if (!dst_on_device)
            LBM_CUDA(cudaMemcpyAsync(dst, conv, (size_t)h->grid.nx * h->grid.ny * 4, cudaMemcpyDeviceToHost, h->stream));
    } else {
        const void *src = which == LBM_FIELD_W ? h->w[h->parity] : h->wd;
        LBM_CUDA(cudaMemcpy2DAsync(dst, row, src, (size_t)h->pitch * h->esize, row, (size_t)h->grid.ny, kind, h->stream));
    }
    if (!dst_on_device) return check_sticky(h);
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_handle *h, int32_t which, const void *src, int32_t src_on_device, int32_t dtype)
{
    lbm::NvtxRange nvtx_("lbm_set_fields");
    if (!h || !src) return fail(LBM_ERR_ARG, "handle or src is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (which != LBM_FIELD_W && which != LBM_FIELD_WDOT) return fail(LBM_ERR_ARG, "unknown field");
    if (dtype != exchange_dtype(h)) return fail(LBM_ERR_ARG, "dtype must be LBM_F64 for F64 storage, LBM_F32 otherwise");
    lbm_status rc = finalize(h);   // the pending crack step reads the fields being replaced
    if (rc != LBM_OK) return rc;
    const size_t row = (size_t)h->grid.nx * h->esize;
    if (which == LBM_FIELD_WDOT && h->esize_d == 0) {
        // leapfrog storage: w_{n-1} = w_n - dt wdot_n, against the current w
        const float *conv = static_cast<const float *>(src);
        if (!src_on_device) {
            LBM_CUDA(cudaMemcpyAsync(h->staging, src, (size_t)h->grid.nx * h->grid.ny * 4, cudaMemcpyHostToDevice, h->stream));
            conv = h->staging;
        }
        LBM_CUDA(launch_lf_set_wdot(static_cast<const float *>(h->w[h->parity]), static_cast<float *>(h->w[h->parity ^ 1]),
                                    h->pitch, h->grid.nx, h->grid.ny, (float)h->grid.dt, conv, h->stream));
    } else if (which == LBM_FIELD_WDOT && wd16(h)) {
        const float *conv = static_cast<const float *>(src);
        if (!src_on_device) {
            LBM_CUDA(cudaMemcpyAsync(h->staging, src, (size_t)h->grid.nx * h->grid.ny * 4, cudaMemcpyHostToDevice, h->stream));
            conv = h->staging;
        }
        LBM_CUDA(wd_from_f32(h, conv, h->wd_scale, h->stream));
    } else {
        void *dst = which == LBM_FIELD_W ? h->w[h->parity] : h->wd;
        LBM_CUDA(cudaMemcpy2DAsync(dst, (size_t)h->pitch * h->esize, src, row, row, (size_t)h->grid.ny,
                                   src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        if (which == LBM_FIELD_W) {
            cudaError_t e = h->esize == 4
                ? launch_fill_pads<float>(static_cast<float *>(dst), h->pitch, h->grid.nx, h->grid.ny, h->grid.edge, h->stream)
                : launch_fill_pads<double>(static_cast<double *>(dst), h->pitch, h->grid.nx, h->grid.ny, h->grid.edge, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "filling pads");
        }
    }
    if (!src_on_device) LBM_CUDA(cudaStreamSynchronize(h->stream));   // pageable source may be reused
    return LBM_OK;
}

// Strided forms: row j of the caller's array starts row_stride elements after
// row j - 1 (row_stride >= nx), e.g. a column window of a wider array.
lbm_status lbm_fields_strided(lbm_handle *h, int32_t which, void *dst, int32_t dst_on_device, int32_t dtype,
                              int64_t row_stride)
{
    lbm::NvtxRange nvtx_("lbm_fields_strided");
    if (!h || !dst) return fail(LBM_ERR_ARG, "handle or dst is NULL");
    if (row_stride < h->grid.nx) return fail(LBM_ERR_ARG, "row_stride must be >= nx");
    if (row_stride == h->grid.nx) return lbm_fields(h, which, dst, dst_on_device, dtype);
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (which != LBM_FIELD_W && which != LBM_FIELD_WDOT) return fail(LBM_ERR_ARG, "unknown field");
    if (dtype != exchange_dtype(h)) return fail(LBM_ERR_ARG, "dtype must be LBM_F64 for F64 storage, LBM_F32 otherwise");
    const size_t row = (size_t)h->grid.nx * h->esize;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const void *src;
    size_t spitch;
    if (which == LBM_FIELD_WDOT && (h->esize_d == 0 || wd16(h))) {
        // converted to a dense FP32 array first (leapfrog: (w_n - w_{n-1}) / dt)
        if (h->esize_d == 0)
            LBM_CUDA(launch_lf_wdot(static_cast<const float *>(h->w[h->parity]), static_cast<const float *>(h->w[h->parity ^ 1]),
                                    h->pitch, h->grid.nx, h->grid.ny, (float)h->grid.dt, h->staging, h->stream));
        else
            LBM_CUDA(wd_to_f32(h, h->staging, h->wd_scale, h->stream));
        src = h->staging;
        spitch = row;
    } else {
        src = which == LBM_FIELD_W ? h->w[h->parity] : h->wd;
        spitch = (size_t)h->pitch * h->esize;
    }
    LBM_CUDA(cudaMemcpy2DAsync(dst, (size_t)row_stride * h->esize, src, spitch, row, (size_t)h->grid.ny, kind, h->stream));
    if (!dst_on_device) return check_sticky(h);
    return LBM_OK;
}

lbm_status lbm_set_fields_strided(lbm_handle *h, int32_t which, const void *src, int32_t src_on_device, int32_t dtype,
                                  int64_t row_stride)
{
    lbm::NvtxRange nvtx_("lbm_set_fields_strided");
    if (!h || !src) return fail(LBM_ERR_ARG, "handle or src is NULL");
    if (row_stride < h->grid.nx) return fail(LBM_ERR_ARG, "row_stride must be >= nx");
    if (row_stride == h->grid.nx) return lbm_set_fields(h, which, src, src_on_device, dtype);
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (which != LBM_FIELD_W && which != LBM_FIELD_WDOT) return fail(LBM_ERR_ARG, "unknown field");
    if (dtype != exchange_dtype(h)) return fail(LBM_ERR_ARG, "dtype must be LBM_F64 for F64 storage, LBM_F32 otherwise");
    const size_t row = (size_t)h->grid.nx * h->esize;
    const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (which == LBM_FIELD_WDOT && (h->esize_d == 0 || wd16(h))) {
        // gathered into a dense FP32 array on the device, then converted as
        // lbm_set_fields converts (which applies the pending crack step first;
        // the staging array is not read by that step)
        LBM_CUDA(cudaMemcpy2DAsync(h->staging, row, src, (size_t)row_stride * h->esize, row, (size_t)h->grid.ny, kind,
                                   h->stream));
        lbm_status rc = lbm_set_fields(h, which, h->staging, 1, dtype);
        if (rc != LBM_OK) return rc;
    } else {
        lbm_status rc = finalize(h);   // the pending crack step reads the fields being replaced
        if (rc != LBM_OK) return rc;
        void *dst = which == LBM_FIELD_W ? h->w[h->parity] : h->wd;
        LBM_CUDA(cudaMemcpy2DAsync(dst, (size_t)h->pitch * h->esize, src, (size_t)row_stride * h->esize, row,
                                   (size_t)h->grid.ny, kind, h->stream));
        if (which == LBM_FIELD_W) {
            cudaError_t e = h->esize == 4
                ? launch_fill_pads<float>(static_cast<float *>(dst), h->pitch, h->grid.nx, h->grid.ny, h->grid.edge, h->stream)
                : launch_fill_pads<double>(static_cast<double *>(dst), h->pitch, h->grid.nx, h->grid.ny, h->grid.edge, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "filling pads");
        }
    }
    if (!src_on_device) LBM_CUDA(cudaStreamSynchronize(h->stream));   // pageable source may be reused
    return LBM_OK;
}

lbm_status lbm_set_wd_scale(lbm_handle *h, double scale)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    int ex = 0;
    if (!(scale > 0.0) || !std::isfinite(scale) || std::frexp(scale, &ex) != 0.5)
        return fail(LBM_ERR_ARG, "the scale must be a positive power of two");
    if (h->lat.storage != LBM_F32_WD_F16) return fail(LBM_ERR_STATE, "only FP16 wdot storage has a scale");
    lbm_status rc = finalize(h);
    if (rc != LBM_OK) return rc;
    LBM_CUDA(wd_to_f32(h, h->staging, h->wd_scale, h->stream));
    LBM_CUDA(wd_from_f32(h, h->staging, scale, h->stream));
    h->wd_scale = scale;
    drop_graph(h);   // the scale is a kernel argument
    h->gen += 1;
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_reset(lbm_handle *h)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    cudaStream_t s = h->stream;
    const size_t mask = (size_t)h->grid.ny * (size_t)h->words * 4;
    LBM_CUDA(cudaMemsetAsync(h->wbase[0], 0, h->plane_bytes, s));
    LBM_CUDA(cudaMemsetAsync(h->wbase[1], 0, h->plane_bytes, s));
    if (h->plane_d_bytes) LBM_CUDA(cudaMemsetAsync(h->wdbase, 0, h->plane_d_bytes, s));
    LBM_CUDA(cudaMemsetAsync(h->cut_h, 0, mask, s));
    LBM_CUDA(cudaMemsetAsync(h->cut_v - h->words, 0, mask + (size_t)h->words * 4, s));   // with the row below row 0
    if (h->line) {
        const size_t n = (size_t)h->grid.ny * h->words;
        LBM_CUDA(cudaMemcpyAsync(h->cut_h, h->init_cut->data(), n * 4, cudaMemcpyHostToDevice, s));
        LBM_CUDA(cudaMemcpyAsync(h->cut_v, h->init_cut->data() + n, n * 4, cudaMemcpyHostToDevice, s));
    } else if (h->cp.mode != CRACK_NONE) {
        LBM_CUDA(cudaMemcpyAsync(h->cut_v + (ptrdiff_t)(h->jc - 1) * h->words, h->init_cut->data(),
                                 h->init_cut->size() * 4, cudaMemcpyHostToDevice, s));
    }
    LBM_CUDA(cudaMemcpyAsync(h->st, &h->init_st, sizeof(CrackState), cudaMemcpyHostToDevice, s));
    LBM_CUDA(launch_wstar(h->st, h->load, h->grid.edge, h->grid.dt, s));
    LBM_CUDA(cudaStreamSynchronize(s));
    h->parity = 0;
    h->pending = false;
    return LBM_OK;
}

lbm_status lbm_set_loading(lbm_handle *h, const lbm_loading *L)
{
    if (!h || !L) return fail(LBM_ERR_ARG, "handle or load is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (L->edge < 0 || L->edge > 3) return fail(LBM_ERR_ARG, "bad load edge");
    if (L->kind < LBM_LOAD_ZERO || L->kind > LBM_LOAD_CONST) return fail(LBM_ERR_ARG, "unknown load kind");
    if (L->kind == LBM_LOAD_SERIES) {
        if (!L->series || L->n_series <= 0) return fail(LBM_ERR_ARG, "series load without data");
        if (L->n_series > h->series_cap[L->edge])
            return fail(LBM_ERR_ARG, "series longer than the one this edge was created with");
    }
    LBM_CUDA(cudaStreamSynchronize(h->stream));   // steps in flight read the old series
    LoadDesc &D = h->load[L->edge];
    if (L->kind == LBM_LOAD_SERIES)
        LBM_CUDA(cudaMemcpyAsync(const_cast<double *>(D.series), L->series, (size_t)L->n_series * 8,
                                 cudaMemcpyHostToDevice, h->stream));
    D.kind = L->kind;
    D.amp = L->amp;
    D.t = L->t_ramp;
    D.n = L->kind == LBM_LOAD_SERIES ? L->n_series : 0;
    // w*(t_n) of the current state follows the new loading
    LBM_CUDA(launch_wstar(h->st + h->parity, h->load, h->grid.edge, h->grid.dt, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    drop_graph(h);   // the loads are kernel arguments
    h->gen += 1;
    return LBM_OK;
}

lbm_status lbm_get_wd_scale(const lbm_handle *h, double *scale)
{
    if (!h || !scale) return fail(LBM_ERR_ARG, "handle or scale is NULL");
    *scale = h->wd_scale;
    return LBM_OK;
}

lbm_status lbm_cut_mask(lbm_handle *h, int32_t which, uint32_t *dst_host, int64_t n_words)
{
    if (!h || !dst_host) return fail(LBM_ERR_ARG, "handle or dst is NULL");
    if (which != LBM_MASK_H && which != LBM_MASK_V) return fail(LBM_ERR_ARG, "unknown mask");
    const int64_t need = (int64_t)h->grid.ny * h->words;
    if (n_words < need) return fail(LBM_ERR_ARG, "dst too small");
    lbm_status rc = finalize(h);
    if (rc != LBM_OK) return rc;
    LBM_CUDA(cudaMemcpyAsync(dst_host, which == LBM_MASK_H ? h->cut_h : h->cut_v, (size_t)need * 4,
                             cudaMemcpyDeviceToHost, h->stream));
    return check_sticky(h);
}

}  // extern "C"

namespace {

// The state of one end of the crack (left: the left end of a two-tip crack)
// and its last records.
lbm_status crack_state_impl(lbm_handle *h, bool left, lbm_crack_state_t *now, double *K_hist, double *v_hist,
                            int64_t *tip_hist, int32_t *npairs_hist, int64_t cap, int64_t *n_written)
{
    lbm::NvtxRange nvtx_("lbm_crack_state");
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (left && !h->cp.two_tips) return fail(LBM_ERR_STATE, "the crack has one growing end");
    lbm_status rc = finalize(h);
    if (rc != LBM_OK) return rc;
    CrackState hs;
    LBM_CUDA(cudaMemcpyAsync(&hs, h->st + h->parity, sizeof hs, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    const TipState &E = left ? hs.l : hs.r;
    int64_t n_cut = hs.i_last >= hs.i_first ? (int64_t)(hs.i_last - hs.i_first + 1) : 0;
    if (h->line && now) {
        // a crack in any direction: the severed links of both masks
        const size_t n = (size_t)h->grid.ny * h->words;
        std::vector<uint32_t> m(2 * n);
        LBM_CUDA(cudaMemcpyAsync(m.data(), h->cut_h, n * 4, cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(cudaMemcpyAsync(m.data() + n, h->cut_v, n * 4, cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(cudaStreamSynchronize(h->stream));
        n_cut = 0;
        for (uint32_t x : m) n_cut += __builtin_popcount(x);
    }
    if (now) {
        now->step = hs.step;
        now->tip_q = E.tip_q;
        now->n_cut = n_cut;
        now->hist_n = hs.hist_n;
        now->tip_x = (double)E.tip_q * kTwoM32 * h->grid.dh;
        now->K = E.K;
        now->v = E.v;
        now->r_min = E.r_min;
        now->npairs = E.npairs;
        now->flags = E.flags;
    }
    int64_t n = 0;
    const int64_t hcap = h->cp.hist_cap;
    if (cap > 0 && hcap > 0) {
        n = hs.hist_n < hcap ? hs.hist_n : hcap;
        if (n > cap) n = cap;
        const int64_t first = hs.hist_n - n;
        std::vector<double> K((size_t)hcap), v((size_t)hcap);
        std::vector<int64_t> tip((size_t)hcap);
        std::vector<int32_t> np((size_t)hcap);
        LBM_CUDA(cudaMemcpyAsync(K.data(), left ? h->hist.Kl : h->hist.K, (size_t)hcap * 8, cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(cudaMemcpyAsync(v.data(), left ? h->hist.vl : h->hist.v, (size_t)hcap * 8, cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(cudaMemcpyAsync(tip.data(), left ? h->hist.tipl : h->hist.tip, (size_t)hcap * 8, cudaMemcpyDeviceToHost,
                                 h->stream));
        LBM_CUDA(cudaMemcpyAsync(np.data(), left ? h->hist.npl : h->hist.np, (size_t)hcap * 4, cudaMemcpyDeviceToHost,
                                 h->stream));
        LBM_CUDA(cudaStreamSynchronize(h->stream));
        for (int64_t q = 0; q < n; ++q) {
            const size_t r = (size_t)((first + q) % hcap);
            if (K_hist) K_hist[q] = K[r];
            if (v_hist) v_hist[q] = v[r];
            if (tip_hist) tip_hist[q] = tip[r];
            if (npairs_hist) npairs_hist[q] = np[r];
        }
    }
    if (n_written) *n_written = n;
    return check_sticky(h);
}

}  // namespace

extern "C" {

lbm_status lbm_crack_state(lbm_handle *h, lbm_crack_state_t *now, double *K_hist, double *v_hist,
                           int64_t *tip_hist, int32_t *npairs_hist, int64_t cap, int64_t *n_written)
{
    return crack_state_impl(h, false, now, K_hist, v_hist, tip_hist, npairs_hist, cap, n_written);
}

lbm_status lbm_crack_state_left(lbm_handle *h, lbm_crack_state_t *now, double *K_hist, double *v_hist,
                                int64_t *tip_hist, int32_t *npairs_hist, int64_t cap, int64_t *n_written)
{
    return crack_state_impl(h, true, now, K_hist, v_hist, tip_hist, npairs_hist, cap, n_written);
}

}  // extern "C"

namespace {

// The tip (left: the start of a two-tip crack) of a crack in any direction
// and the y of its last records.
lbm_status line_tip_impl(lbm_handle *h, bool left, int64_t *x_q, int64_t *y_q, int64_t *y_hist, int64_t cap,
                         int64_t *n_written)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (!h->line) return fail(LBM_ERR_STATE, "the handle has no crack in any direction");
    if (left && !h->cp.two_tips) return fail(LBM_ERR_STATE, "the crack has one growing end");
    lbm_status rc = finalize(h);
    if (rc != LBM_OK) return rc;
    CrackState hs;
    LBM_CUDA(cudaMemcpyAsync(&hs, h->st + h->parity, sizeof hs, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    const TipState &E = left ? hs.l : hs.r;
    if (x_q) *x_q = E.tip_q;
    if (y_q) *y_q = E.tip_yq;
    int64_t n = 0;
    const int64_t hcap = h->cp.hist_cap;
    if (y_hist && cap > 0 && hcap > 0) {
        n = hs.hist_n < hcap ? hs.hist_n : hcap;
        if (n > cap) n = cap;
        const int64_t first = hs.hist_n - n;
        std::vector<int64_t> ty((size_t)hcap);
        LBM_CUDA(cudaMemcpyAsync(ty.data(), left ? h->hist.tipyl : h->hist.tipy, (size_t)hcap * 8,
                                 cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA(cudaStreamSynchronize(h->stream));
        for (int64_t q = 0; q < n; ++q) y_hist[q] = ty[(size_t)((first + q) % hcap)];
    }
    if (n_written) *n_written = n;
    return check_sticky(h);
}

}  // namespace

extern "C" {

lbm_status lbm_line_tip(lbm_handle *h, int64_t *x_q, int64_t *y_q, int64_t *y_hist, int64_t cap, int64_t *n_written)
{
    return line_tip_impl(h, false, x_q, y_q, y_hist, cap, n_written);
}

lbm_status lbm_line_tip_left(lbm_handle *h, int64_t *x_q, int64_t *y_q, int64_t *y_hist, int64_t cap,
                             int64_t *n_written)
{
    return line_tip_impl(h, true, x_q, y_q, y_hist, cap, n_written);
}

lbm_status lbm_sync(lbm_handle *h)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    return check_sticky(h);
}

lbm_status lbm_set_stream(lbm_handle *h, void *stream)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    h->stream = (cudaStream_t)stream;
    return LBM_OK;
}

lbm_status lbm_set_launch(lbm_handle *h, int32_t band_rows)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (band_rows < 0 || band_rows > (1 << 20)) return fail(LBM_ERR_ARG, "band_rows out of range");
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    drop_graph(h);
    if (h->line) {
        // the march blocks of a crack in any direction: bands of band_rows
        // rows (every kernel computes its grid and its blocks' rows from it)
        h->cp.band = band_rows > 0 ? std::min(band_rows, h->grid.ny) : h->line_band0;
        h->gen += 1;
        clear_error();
        return LBM_OK;
    }
    return plan_bands(h, band_rows);
}

lbm_status lbm_set_bulk(lbm_handle *h, int32_t enable)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    const bool on = enable != 0 && h->esize == 4 && !h->line && h->q == 5;
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    int bps = 0;
    LBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, step_kernel_for(h->lat.storage, on), kThreads, 0));
    if (bps < 1) return fail(LBM_ERR_ARG, "the step kernel does not fit on an SM");
    h->bulk = on;
    h->bps = bps;
    drop_graph(h);
    lbm_status rc = plan_bands(h, 0);
    if (rc == LBM_OK) clear_error();
    return rc;
}

lbm_status lbm_set_chained(lbm_handle *h, int32_t enable)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    h->chained = enable != 0;
    drop_graph(h);
    clear_error();
    return LBM_OK;
}

lbm_status lbm_set_face_solve(lbm_handle *h, int32_t mode, int32_t *chunked)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (mode != 0 && mode != 1) return fail(LBM_ERR_ARG, "mode must be 0 (chunked where possible) or 1 (one CTA)");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    h->face_solve = mode;
    drop_graph(h);
    h->gen += 1;
    if (chunked) *chunked = (h->n_face_chunks > 0 && mode == 0) ? 1 : 0;
    clear_error();
    return LBM_OK;
}

lbm_status lbm_get_launch(const lbm_handle *h, int32_t *band_rows, int32_t *ctas, int32_t *threads,
                          int32_t *ctas_per_sm)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (band_rows) *band_rows = h->line ? h->cp.band : h->band_rows;
    if (ctas)
        *ctas = h->line ? 1 + h->ncb * ((h->grid.ny + h->cp.band - 1) / h->cp.band)
                        : h->n_bands * h->ncb;
    if (threads) *threads = kThreads;
    if (ctas_per_sm) *ctas_per_sm = h->bps;
    return LBM_OK;
}

lbm_status lbm_set_profiling(lbm_handle *h, int32_t enable)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    if (enable && !h->ev) {
        h->ev = new (std::nothrow) std::vector<cudaEvent_t>(2 * 1024);
        h->ev_kind = new (std::nothrow) std::vector<int>(1024);
        if (!h->ev || !h->ev_kind) return fail(LBM_ERR_OOM, "host allocation failed");
        for (auto &e : *h->ev) {
            cudaError_t ce = cudaEventCreate(&e);
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventCreate");
        }
        h->ev_used = 0;
    }
    if (!enable && h->ev) LBM_CUDA(drain_profile(h));
    h->profiling = enable ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_handle *h, double *step_ms, int64_t *n_step, double *finalize_ms, int64_t *n_finalize,
                            int32_t reset)
{
    if (!h) return fail(LBM_ERR_ARG, "handle is NULL");
    LBM_CUDA(drain_profile(h));
    if (step_ms) *step_ms = h->step_ms;
    if (n_step) *n_step = h->n_step;
    if (finalize_ms) *finalize_ms = h->fin_ms;
    if (n_finalize) *n_finalize = h->n_fin;
    if (reset) {
        h->step_ms = h->fin_ms = 0.0;
        h->n_step = h->n_fin = 0;
    }
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------- copy-out of 16-bit wdot, no allocation
//
// The conversion of a 16-bit wdot plane to FP32 normally goes through the
// handle's staging buffer (allocated by lbm_create).  lbm_wdot_to_host_noalloc
// runs the same conversion kernel into one fixed device array that belongs to
// the library, so it allocates nothing and leaves the handle's staging buffer
// alone.  Nothing in the array needs to start at zero: a call reads back only
// elements it has just written.  All calls on a device share the array, so
// calls that overlap in time (from several threads, or on several streams)
// race on it; callers serialise them.  Like every call on a handle, it must
// also be serialised with the other calls on the same handle (it applies the
// pending crack step and enqueues work on the handle's stream).

namespace {

constexpr int64_t kNoAllocFloats = (int64_t)1 << 20;   // 4 MiB: lattices of up to 2^20 sites
constexpr int kNoAllocDevices = 64;

static __device__ __align__(256) float g_noalloc_wd[kNoAllocFloats];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocDevices];

// Address of the array on the current device.  It is looked up again on
// every call made outside a stream capture (the module can load at another
// address after the device's primary context is torn down and re-created);
// during a capture, where the lookup is not allowed, the address of the last
// lookup on this device is used, so a first call on a device must not come
// while its stream is being captured.
cudaError_t noalloc_scratch(cudaStream_t s, float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_wd);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    } else if (!g_noalloc_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = static_cast<float *>(g_noalloc_addr[dev]);
    return cudaSuccess;
}

}  // namespace

extern "C" {

lbm_status lbm_wdot_to_host_noalloc(lbm_handle *h, float *dst_host, int64_t n_floats)
{
    if (!h || !dst_host) return fail(LBM_ERR_ARG, "handle or dst is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    if (!wd16(h)) return fail(LBM_ERR_STATE, "only 16-bit wdot storage is converted; use lbm_fields");
    const int64_t n = (int64_t)h->grid.nx * h->grid.ny;
    if (n > kNoAllocFloats) return fail(LBM_ERR_ARG, "lattice larger than the fixed conversion array (2^20 sites)");
    if (n_floats < n) return fail(LBM_ERR_ARG, "dst too small");
    float *scratch = nullptr;
    LBM_CUDA(noalloc_scratch(h->stream, &scratch));
    // the pending crack step goes first, in the stream order lbm_fields uses
    // (it changes only the masks and the crack state, not wdot; check_sticky
    // below would otherwise apply it after the copy)
    lbm_status rc = finalize(h);
    if (rc != LBM_OK) return rc;
    LBM_CUDA(wd_to_f32(h, scratch, h->wd_scale, h->stream));
    LBM_CUDA(cudaMemcpyAsync(dst_host, scratch, (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream));
    return check_sticky(h);
}

}  // extern "C"

namespace {

// Checkpoint file: this header, then the w plane, the stored wdot plane, the
// two cut masks, the crack state and the history ring of each end, as raw
// bytes in that order.
struct CkptHeader {
    char magic[8];
    int32_t version, crack_state_bytes;
    lbm_grid grid;
    lbm_lattice lat;
    lbm_material mat;
    lbm_crack crack;
    int32_t load_kind[4];
    double load_amp[4], load_t[4];
    int64_t load_n[4];
    int64_t pitch, plane_bytes, plane_d_bytes, mask_bytes, hist_cap, hist_cap_l;
    int32_t words, ny;
    double wd_scale;
};
constexpr char kCkptMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};

void ckpt_header(const lbm_handle *h, CkptHeader &c)
{
    std::memset(&c, 0, sizeof c);
    std::memcpy(c.magic, kCkptMagic, 8);
    c.version = 2;
    c.crack_state_bytes = (int32_t)sizeof(CrackState);
    c.grid = h->grid;
    c.lat = h->lat;
    c.mat = h->mat;
    c.crack = h->crack;
    for (int e = 0; e < 4; ++e) {
        c.load_kind[e] = h->load[e].kind;
        c.load_amp[e] = h->load[e].amp;
        c.load_t[e] = h->load[e].t;
        c.load_n[e] = h->load[e].n;
    }
    c.pitch = h->pitch;
    c.plane_bytes = (int64_t)h->plane_bytes;
    // leapfrog storage: the second plane is w_{n-1}
    c.plane_d_bytes = (int64_t)(h->esize_d ? h->plane_d_bytes : h->plane_bytes);
    c.mask_bytes = (int64_t)h->grid.ny * h->words * 4;
    c.hist_cap = h->cp.mode != CRACK_NONE ? h->cp.hist_cap : 1;
    c.hist_cap_l = h->cp.two_tips ? c.hist_cap : 1;
    c.words = h->words;
    c.ny = h->grid.ny;
    c.wd_scale = h->wd_scale;
}

// Every field but the wdot scale (which the checkpoint carries) must agree.
bool ckpt_compatible(const CkptHeader &a, const CkptHeader &b)
{
    CkptHeader x = a, y = b;
    x.wd_scale = y.wd_scale = 0.0;
    return std::memcmp(&x, &y, sizeof x) == 0;
}

// The device buffers of a checkpoint, in file order, with their sizes.
std::vector<std::pair<void *, size_t>> ckpt_buffers(lbm_handle *h, const CkptHeader &c)
{
    const History &H = h->hist;
    return {{h->wbase[h->parity], (size_t)c.plane_bytes},
            {h->esize_d ? h->wdbase : h->wbase[h->parity ^ 1], (size_t)c.plane_d_bytes},
            {h->cut_h, (size_t)c.mask_bytes},
            {h->cut_v - h->words, (size_t)c.mask_bytes + (size_t)c.words * 4},   // with the row below row 0
            {h->st + h->parity, sizeof(CrackState)},
            {H.K, (size_t)c.hist_cap * 8},
            {H.v, (size_t)c.hist_cap * 8},
            {H.tip, (size_t)c.hist_cap * 8},
            {H.np, (size_t)c.hist_cap * 4},
            {H.Kl, (size_t)c.hist_cap_l * 8},
            {H.vl, (size_t)c.hist_cap_l * 8},
            {H.tipl, (size_t)c.hist_cap_l * 8},
            {H.npl, (size_t)c.hist_cap_l * 4},
            {H.tipy, (size_t)(h->line ? c.hist_cap : 1) * 8},
            {H.tipyl, (size_t)(h->line ? c.hist_cap_l : 1) * 8}};
}

}  // namespace

extern "C" {

lbm_status lbm_save(lbm_handle *h, const char *path)
{
    lbm::NvtxRange nvtx_("lbm_save");
    if (!h || !path) return fail(LBM_ERR_ARG, "handle or path is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    lbm_status rc = finalize(h);   // the state after the crack step of the last time step
    if (rc != LBM_OK) return rc;
    CkptHeader c;
    ckpt_header(h, c);
    const auto bufs = ckpt_buffers(h, c);
    std::vector<std::vector<char>> host(bufs.size());
    for (size_t q = 0; q < bufs.size(); ++q) {
        host[q].resize(bufs[q].second);
        LBM_CUDA(cudaMemcpyAsync(host[q].data(), bufs[q].first, bufs[q].second, cudaMemcpyDeviceToHost, h->stream));
    }
    rc = check_sticky(h);   // synchronises the stream
    if (rc != LBM_OK) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(LBM_ERR_IO, std::string("cannot open ") + path + " for writing");
    bool ok = std::fwrite(&c, sizeof c, 1, f) == 1;
    for (size_t q = 0; ok && q < host.size(); ++q) ok = std::fwrite(host[q].data(), 1, host[q].size(), f) == host[q].size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(LBM_ERR_IO, std::string("writing ") + path + " failed");
    return LBM_OK;
}

lbm_status lbm_load(lbm_handle *h, const char *path)
{
    lbm::NvtxRange nvtx_("lbm_load");
    if (!h || !path) return fail(LBM_ERR_ARG, "handle or path is NULL");
    if (h->sticky != LBM_OK) return fail(h->sticky, "the handle is in an error state");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    CkptHeader c, mine;
    if (std::fread(&c, sizeof c, 1, f) != 1 || std::memcmp(c.magic, kCkptMagic, 8) != 0 || c.version != 2) {
        std::fclose(f);
        return fail(LBM_ERR_IO, std::string(path) + " is not a lattice checkpoint");
    }
    ckpt_header(h, mine);
    if (!ckpt_compatible(c, mine)) {
        std::fclose(f);
        return fail(LBM_ERR_ARG, "the checkpoint was written by a lattice of another configuration");
    }
    const auto bufs = ckpt_buffers(h, mine);
    std::vector<std::vector<char>> host(bufs.size());
    bool ok = true;
    for (size_t q = 0; ok && q < bufs.size(); ++q) {
        host[q].resize(bufs[q].second);
        ok = std::fread(host[q].data(), 1, host[q].size(), f) == host[q].size();
    }
    std::fclose(f);
    if (!ok) return fail(LBM_ERR_IO, std::string(path) + " is truncated");
    cudaError_t e = cudaStreamSynchronize(h->stream);   // no step may be in flight on the buffers
    if (e != cudaSuccess) return cuda_fail(e, "synchronising before the load");
    for (size_t q = 0; q < bufs.size(); ++q)
        LBM_CUDA(cudaMemcpyAsync(bufs[q].first, host[q].data(), bufs[q].second, cudaMemcpyHostToDevice, h->stream));
    h->pending = false;               // the saved state had its crack step applied
    if (h->wd_scale != c.wd_scale) {
        h->wd_scale = c.wd_scale;
        drop_graph(h);                // the scale is a kernel argument
    }
    return check_sticky(h);           // synchronises: the host buffers go out of scope
}

lbm_status lbm_device_bytes(const lbm_handle *h, int64_t *bytes)
{
    if (!h || !bytes) return fail(LBM_ERR_ARG, "handle or bytes is NULL");
    *bytes = (int64_t)h->block_bytes;
    return LBM_OK;
}

void lbm_destroy(lbm_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->ev) {
        for (auto &e : *h->ev) cudaEventDestroy(e);
        delete h->ev;
        delete h->ev_kind;
    }
    dev_free(h, h->faces);
    dev_free(h, h->face_scratch);
    dev_free(h, h->block);
    free_host(h);
}

// ---------------------------------------------------------------- batches

}  // extern "C"

struct lbm_batch {
    std::vector<lbm_handle *> hs;
    int storage;
    void *block;         // descriptors (2 per lattice: parity 0, 1) then units
    size_t block_bytes;
    void *descs;
    BatchUnit *units;
    int n_units;
    BatchUnit *eunits;   // edge-rule units: 128 edge sites of one lattice (LBM_BC_MACROSCOPIC_EDGES)
    int n_eunits;
    int q;               // velocity set of every member (5: D2Q5, 9: D2Q9)
    bool line;           // every member has a crack in any direction (lbm_create_line)
    BatchUnit *funits;   // D2Q9 crack-face units: 128 columns of one lattice with macroscopic crack faces
    int n_funits;
    BatchPiece *pieces;  // balanced step (band_rows = -1): the pieces of every CTA ...
    int32_t *poff;       // ... CTA c runs pieces poff[c] .. poff[c + 1] - 1
    int n_pcta;          // CTAs of the balanced step (0: the per-band launch)
    int threads;         // threads per CTA: column blocks of threads 16-byte vectors
    int band_rows;       // rows per band (the crack sub-bands have their own height); -1: balanced
    int lookahead;       // rows of loads the march keeps ahead (1 or 2)
    bool chained;        // each step's launches chained by programmatic dependent launch
    bool persistent;     // lbm_batch_step as one cooperative launch (grid barrier between steps)
    long long budget;    // clock64 cycles a CTA waits at that barrier before giving up
    GridBarrier *bar;    // the barrier (own allocation, with the batch's error word after it)
    uint32_t *err;
    lbm_allocator alloc;
    bool custom_alloc;
    cudaStream_t stream;
    cudaStream_t cap_stream;
    ChunkGraph graph;    // graphs of runs of batched steps
    bool owns;           // made by lbm_create_batch: the member handles are destroyed with the batch
};

namespace {

// Edge-rule units of the lattices with the macroscopic rule on their outer
// edges: 128 edge sites each (the batch step applies it after the update).
template <typename T, typename D>
void edge_units(const lbm_batch *b, std::vector<BatchUnit> &out)
{
    for (size_t i = 0; i < b->hs.size(); ++i) {
        if (!b->hs[i]->edge_macro) continue;
        StepArgs<T, D> a;
        make_step_args(b->hs[i], 0, a);
        const int n = edge_rule_count(a);
        for (int t0 = 0; t0 < n; t0 += 128) {
            BatchUnit u;
            u.inst = (int32_t)i;
            u.cb = t0;
            u.band = 0;
            u.pad = 0;
            out.push_back(u);
        }
    }
}

template <typename T, typename D>
void fill_descs(const lbm_batch *b, std::vector<char> &buf)
{
    buf.resize(2 * b->hs.size() * sizeof(StepArgs<T, D>));
    StepArgs<T, D> *d = reinterpret_cast<StepArgs<T, D> *>(buf.data());
    for (size_t i = 0; i < b->hs.size(); ++i) {
        make_step_args(b->hs[i], 0, d[2 * i]);
        make_step_args(b->hs[i], 1, d[2 * i + 1]);
    }
}

template <typename T, typename D>
cudaError_t enqueue_batch_persistent_t(const lbm_batch *b, int par, int64_t n, cudaStream_t s)
{
    const StepArgs<T, D> *d = static_cast<const StepArgs<T, D> *>(b->descs);
    cudaError_t e = cudaMemsetAsync(b->bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    return launch_batch_persistent(d, (int)b->hs.size(), b->units, b->n_units, b->eunits, b->n_eunits, par, n, b->bar,
                                   b->err, b->budget, b->threads, s);
}

cudaError_t enqueue_batch_persistent(const lbm_batch *b, int par, int64_t n, cudaStream_t s)
{
    switch (b->storage) {
    case LBM_F32: return enqueue_batch_persistent_t<float, float>(b, par, n, s);
    case LBM_F32_WD_BF16: return enqueue_batch_persistent_t<float, __nv_bfloat16>(b, par, n, s);
    case LBM_F32_WD_F16: return enqueue_batch_persistent_t<float, __half>(b, par, n, s);
    case LBM_F32_LEAPFROG: return enqueue_batch_persistent_t<float, Lf>(b, par, n, s);
    default: return enqueue_batch_persistent_t<double, double>(b, par, n, s);
    }
}

template <typename T, typename D>
cudaError_t enqueue_batch_step_t(const lbm_batch *b, int par, cudaStream_t s)
{
    const StepArgs<T, D> *d = static_cast<const StepArgs<T, D> *>(b->descs);
    if constexpr (!std::is_same<D, Lf>::value) {   // a crack in any direction has no leapfrog storage
        if (b->line) {
            // the batched line step, then the face rule of each lattice with
            // macroscopic faces (its own launch, as for the lattice alone)
            cudaError_t e = launch_batch_line(d, b->units, b->n_units, par, s, b->chained);
            for (const lbm_handle *h : b->hs) {
                if (e != cudaSuccess) break;
                if (h->n_face_chunks == 0 && h->n_faces == 0) continue;
                StepArgs<T, D> a;
                make_step_args(h, par, a);
                a.chained = b->chained ? 1 : 0;
                if (h->n_face_chunks > 0 && h->face_solve == 0)
                    e = launch_line_faces_chunked(a, h->face_chunks, h->n_face_chunks, h->face_items, s);
                else if (h->n_faces > 0)
                    e = launch_line_faces(a, h->faces, h->n_faces, h->face_scratch, s);
            }
            return e;
        }
    }
    if constexpr (std::is_same<T, D>::value) {
        if (b->q == 9) {
            cudaError_t e = launch_batch_d2q9(d, b->units, b->n_units, b->funits, b->n_funits, par, s, b->chained);
            if (e == cudaSuccess && b->n_eunits > 0)
                e = launch_batch_edge_rule(d, b->eunits, b->n_eunits, par, s, b->chained);
            return e;
        }
    }
    cudaError_t e = b->n_pcta > 0
                        ? launch_batch_pieces(d, b->pieces, b->poff, b->n_pcta, par, s, b->threads, b->lookahead,
                                              b->chained)
                        : launch_batch_step(d, b->units, b->n_units, par, s, b->threads, b->lookahead, b->chained);
    if (e == cudaSuccess && b->n_eunits > 0) e = launch_batch_edge_rule(d, b->eunits, b->n_eunits, par, s, b->chained);
    return e;
}

cudaError_t enqueue_batch_step(const lbm_batch *b, int par, cudaStream_t s)
{
    switch (b->storage) {
    case LBM_F32: return enqueue_batch_step_t<float, float>(b, par, s);
    case LBM_F32_WD_BF16: return enqueue_batch_step_t<float, __nv_bfloat16>(b, par, s);
    case LBM_F32_WD_F16: return enqueue_batch_step_t<float, __half>(b, par, s);
    case LBM_F32_LEAPFROG: return enqueue_batch_step_t<float, Lf>(b, par, s);
    default: return enqueue_batch_step_t<double, double>(b, par, s);
    }
}

// The batched step kernel for a storage, CTA width and lookahead (for
// occupancy queries).
cudaError_t batch_kernel_ptr(int storage, int threads, int la, const void **fn)
{
    switch (storage) {
    case LBM_F32: return batch_step_kernel_ptr<float, float>(threads, la, fn);
    case LBM_F32_WD_BF16: return batch_step_kernel_ptr<float, __nv_bfloat16>(threads, la, fn);
    case LBM_F32_WD_F16: return batch_step_kernel_ptr<float, __half>(threads, la, fn);
    case LBM_F32_LEAPFROG: return batch_step_kernel_ptr<float, Lf>(threads, la, fn);
    default: return batch_step_kernel_ptr<double, double>(threads, la, fn);
    }
}

cudaError_t batch_piece_ptr(int storage, int threads, int la, const void **fn)
{
    switch (storage) {
    case LBM_F32: return batch_piece_kernel_ptr<float, float>(threads, la, fn);
    case LBM_F32_WD_BF16: return batch_piece_kernel_ptr<float, __nv_bfloat16>(threads, la, fn);
    case LBM_F32_WD_F16: return batch_piece_kernel_ptr<float, __half>(threads, la, fn);
    case LBM_F32_LEAPFROG: return batch_piece_kernel_ptr<float, Lf>(threads, la, fn);
    default: return batch_piece_kernel_ptr<double, double>(threads, la, fn);
    }
}

void batch_release_block(lbm_batch *b)
{
    if (!b->block) return;
    cudaStreamSynchronize(b->stream);
    if (b->custom_alloc) b->alloc.release(b->block, b->alloc.ctx);
    else cudaFree(b->block);
    b->block = nullptr;
    b->block_bytes = 0;
}

void *batch_alloc(lbm_batch *b, size_t bytes)
{
    void *p = nullptr;
    if (b->custom_alloc) p = b->alloc.alloc(bytes, b->alloc.ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    return p;
}

void batch_free(lbm_batch *b, void *p)
{
    if (!p) return;
    if (b->custom_alloc) b->alloc.release(p, b->alloc.ctx);
    else cudaFree(p);
}

// Band heights of a batch whose CTAs all fit in one wave (rows = 0): every
// lattice's bands about equally tall, as tall as the resident slots allow,
// so each CTA marches a long band (few halo rows) and no second wave or tail
// of short units follows.  Returns per lattice the height to partition with.
lbm_status batch_one_wave(lbm_batch *b, int threads, int la, std::vector<int> &heights)
{
    const void *fn = nullptr;
    cudaError_t e = batch_kernel_ptr(b->storage, threads, la, &fn);
    if (e != cudaSuccess) return cuda_fail(e, "selecting the batch kernel");
    int bps = 0;
    LBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, 0));
    const int64_t slots = (int64_t)b->hs[0]->sms * std::max(bps, 1);
    heights.assign(b->hs.size(), 1);
    // strip-rows: column blocks x rows, the crack sub-bands apart
    int64_t total = 0;
    int64_t crack_units = 0;
    std::vector<int> ncb(b->hs.size()), body(b->hs.size());
    for (size_t i = 0; i < b->hs.size(); ++i) {
        const lbm_handle *h = b->hs[i];
        const int cols = threads * (int)(16 / h->esize);
        ncb[i] = (h->grid.nx + cols - 1) / cols;
        const bool crack = h->cp.mode != CRACK_NONE && !h->cp.line;
        const int hh = !crack ? 0 : (h->cp.macro ? 3 : 1);
        const int nsub = !crack ? 0 : ((h->jc >= hh ? 1 : 0) + (h->jc + hh <= h->grid.ny ? 1 : 0));
        body[i] = h->grid.ny - nsub * hh;
        total += (int64_t)ncb[i] * body[i];
        crack_units += (int64_t)ncb[i] * nsub;
    }
    const int64_t free_slots = std::max<int64_t>(slots - crack_units, 1);
    for (int64_t target = std::max<int64_t>(1, (total + free_slots - 1) / free_slots);; ++target) {
        int64_t units = crack_units;
        for (size_t i = 0; i < b->hs.size(); ++i) {
            const int nb = std::max<int64_t>(1, (body[i] + target / 2) / target);
            const int rows = (body[i] + nb - 1) / nb;
            heights[i] = std::max(rows, 1);
            units += (int64_t)ncb[i] * ((body[i] + heights[i] - 1) / heights[i] + 2);   // + pieces around the crack
        }
        if (units <= slots || target > 1 << 20) break;
    }
    return LBM_OK;
}

// The pieces of the balanced step (band_rows = -1).  Every lattice keeps its
// band table (bands of 16 rows; the crack sub-bands are units of their own,
// as in the per-band launch); the rows outside the crack sub-bands are cut
// into row blocks about as tall as one CTA's share of all rows, column block
// by column block, and this sequence (lattice by lattice, row block by row
// block, column block by column block, a lattice's crack sub-band units
// after its rows below the crack) is cut into one contiguous run per CTA of
// equal weight (a row of a column block weighs 1, a crack sub-band unit its
// rows plus four, for the loads it issues at once and the crack step).  So
// every CTA marches about the same number of rows whatever the lattices'
// heights, the CTAs of horizontally adjacent column blocks march the same
// rows at about the same time (their halo columns meet in L2), and a piece
// that would leave fewer than four rows of its row block is given them.
lbm_status batch_plan_pieces(lbm_batch *b, int threads, int la, std::vector<BatchPiece> &pieces,
                             std::vector<int32_t> &off)
{
    const void *fn = nullptr;
    cudaError_t e = batch_piece_ptr(b->storage, threads, la, &fn);
    if (e != cudaSuccess) return cuda_fail(e, "selecting the balanced batch kernel");
    int bps = 0;
    LBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, 0));
    const int64_t slots = (int64_t)b->hs[0]->sms * std::max(bps, 1);
    struct Item {
        int32_t inst, cb, j0, j1, duty, weight;
    };
    // first pass: the number of CTAs (at least 16 rows each) and a CTA's share
    int64_t weight = 0;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        const lbm_handle *h = b->hs[i];
        const int cols = threads * (int)(16 / h->esize);
        const int ncb = (h->grid.nx + cols - 1) / cols;
        const int hh = h->crack_band < 0 ? 0 : (h->cp.macro ? 3 : 1);
        const int nsub = h->crack_band < 0 ? 0 : (h->cp.sides == 3 ? 2 : 1);
        weight += (int64_t)ncb * (h->grid.ny - nsub * hh) + (int64_t)ncb * nsub * (hh + 4);
    }
    const int64_t n_cta = std::max<int64_t>(1, std::min<int64_t>(slots, weight / 16));
    const double share = (double)weight / (double)n_cta;
    std::vector<Item> seq;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        const lbm_handle *h = b->hs[i];
        const std::vector<Unit> &U = *h->units_h;
        const int cols = threads * (int)(16 / h->esize);
        const int ncb = (h->grid.nx + cols - 1) / cols;
        if (ncb > 32767) return fail(LBM_ERR_ARG, "lattice too wide for the balanced batch");
        const int cband = h->crack_band;
        const int hh = cband < 0 ? 0 : (h->cp.macro ? 3 : 1);
        const int nsub = cband < 0 ? 0 : (h->cp.sides == 3 ? 2 : 1);
        auto is_crack = [&](int band) { return cband >= 0 && (band == cband || (band == cband + 1 && nsub == 2)); };
        // the band that carries the per-step state duty in the per-band launch
        const int dband = cband < 0 ? 0 : (h->n_bands > 2 ? (cband > 0 ? 0 : cband + nsub) : -1);
        const int dkind = cband < 0 ? 1 : 2;
        int band = 0;
        while (band < h->n_bands) {
            if (is_crack(band)) {
                for (int cb = 0; cb < ncb; ++cb) seq.push_back({(int32_t)i, cb, -(band + 1), 0, 0, hh + 4});
                ++band;
                continue;
            }
            const int r0 = U[band].j0;
            int r1 = U[band].j1;
            const bool duty_here = band == dband;
            ++band;
            while (band < h->n_bands && !is_crack(band)) r1 = U[band++].j1;
            // row blocks of about one CTA's share
            const int H = r1 - r0;
            const int nblk = std::max(1, (int)std::lround((double)H / std::max(share, 1.0)));
            for (int k = 0; k < nblk; ++k) {
                const int a0 = r0 + (int)((int64_t)H * k / nblk), a1 = r0 + (int)((int64_t)H * (k + 1) / nblk);
                if (a1 <= a0) continue;
                for (int cb = 0; cb < ncb; ++cb)
                    seq.push_back({(int32_t)i, cb, a0, a1, (k == 0 && cb == 0 && duty_here) ? dkind : 0, a1 - a0});
            }
        }
    }
    // cut the sequence into n_cta runs, each about the weight left over the
    // CTAs left (so that short runs early on do not pile work on the last)
    pieces.clear();
    off.assign(1, 0);
    int64_t c = 0;
    double load = 0.0, left = (double)weight;
    double target = left / (double)n_cta;
    auto next_cta = [&]() {
        off.push_back((int32_t)pieces.size());
        left -= load;
        load = 0.0;
        ++c;
        target = left / (double)(n_cta - c);
    };
    for (const Item &it : seq) {
        if (it.j0 < 0) {
            if (load > 0.0 && load + 0.5 * it.weight > target && c < n_cta - 1) next_cta();
            pieces.push_back({it.inst, (int16_t)it.cb, 0, it.j0, it.j1});
            load += it.weight;
            continue;
        }
        int r = it.j0;
        bool first = true;
        while (r < it.j1) {
            if (load > 0.0 && load >= target - 0.5 && c < n_cta - 1) next_cta();
            int take = c == n_cta - 1 ? it.j1 - r : std::max(1, (int)std::ceil(target - load - 1e-9));
            take = std::min(take, it.j1 - r);
            if (it.j1 - r - take < 4) take = it.j1 - r;   // no sliver of under four rows left behind
            if (take < 4 && load > 0.0 && c < n_cta - 1 && it.j1 - r >= 4) {
                next_cta();   // nor a piece of under four rows at a run's end
                continue;
            }
            pieces.push_back({it.inst, (int16_t)it.cb, (int16_t)(first ? it.duty : 0), r, r + take});
            first = false;
            r += take;
            load += take;
        }
    }
    while (c < n_cta) next_cta();
    if ((int64_t)off.size() != n_cta + 1) return fail(LBM_ERR_ARG, "balanced batch: inconsistent piece table");
    return LBM_OK;
}

// Re-partition every lattice into bands of `rows` rows (0: the single-wave
// heights of batch_one_wave) and rebuild the unit table for CTAs of
// `threads` threads (column blocks of threads 16-byte vectors) and the
// descriptor table, for a march with `la` rows of lookahead; the block
// grows when the tables do.
lbm_status batch_build(lbm_batch *b, int threads, int rows, int la)
{
    if (threads != 32 && threads != 64 && threads != kThreads)
        return fail(LBM_ERR_ARG, "threads per CTA must be 32, 64 or 128");
    if (rows < -2) return fail(LBM_ERR_ARG, "band_rows must be >= 0, -1 (balanced) or -2 (tapered)");
    if (la != 1 && la != 2) return fail(LBM_ERR_ARG, "lookahead must be 1 or 2 rows");
    if (b->q == 9 && (threads != kThreads || la != 1 || rows == -1))
        return fail(LBM_ERR_ARG, "a D2Q9 batch takes CTAs of 128 threads, bands (not the balanced form) and a lookahead of one row");
    if (b->line && (threads != kThreads || la != 1 || rows < 0))
        return fail(LBM_ERR_ARG, "a batch of cracks in any direction takes CTAs of 128 threads and a lookahead of one row");
    const bool balanced = rows == -1;
    // the balanced step keeps bands of 16 rows for its crack sub-bands and for
    // the persistent form
    std::vector<int> heights(b->hs.size(), balanced ? 16 : rows);
    if (rows == 0) {
        lbm_status rc = batch_one_wave(b, threads, la, heights);
        if (rc != LBM_OK) return rc;
    }
    // the order the lattices' units are launched in
    std::vector<size_t> order(b->hs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    if (rows == -2) {
        // tapered: the lattices by size, largest first; bands of 48 rows
        // (few halo rows) until the smallest lattices that hold the last
        // sixth of the sites, which take bands of 8 rows, so that the units
        // the dispatcher hands out last are short and the step ends with a
        // short tail
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
            return (int64_t)b->hs[x]->grid.nx * b->hs[x]->grid.ny > (int64_t)b->hs[y]->grid.nx * b->hs[y]->grid.ny;
        });
        int64_t total = 0, seen = 0;
        for (const lbm_handle *h : b->hs) total += (int64_t)h->grid.nx * h->grid.ny;
        for (size_t k = 0; k < order.size(); ++k) {
            const lbm_handle *h = b->hs[order[k]];
            heights[order[k]] = seen * 6 < total * 5 ? 48 : 8;
            seen += (int64_t)h->grid.nx * h->grid.ny;
        }
    }
    std::vector<BatchUnit> units;
    if (b->line) {
        // each lattice keeps its own line-step grid: block 0 the tip CTA, then
        // its march blocks (bands of the lattice's fixed height)
        for (size_t i = 0; i < b->hs.size(); ++i) {
            lbm_handle *h = b->hs[i];
            drop_graph(h);
            const int n = 1 + h->ncb * ((h->grid.ny + h->cp.band - 1) / h->cp.band);
            for (int u = 0; u < n; ++u) units.push_back(BatchUnit{(int32_t)i, u, 0, 0});
        }
    } else {
        for (size_t i : order) {
            lbm_handle *h = b->hs[i];
            drop_graph(h);
            lbm_status rc = plan_bands(h, heights[i]);
            if (rc != LBM_OK) return rc;
            const int cols = threads * (int)(16 / h->esize);
            const int ncb = (h->grid.nx + cols - 1) / cols;
            for (int band = 0; band < h->n_bands; ++band)
                for (int cb = 0; cb < ncb; ++cb) {
                    BatchUnit u;
                    u.inst = (int32_t)i;
                    u.cb = cb;
                    u.band = band;
                    u.pad = 0;
                    units.push_back(u);
                }
        }
    }
    std::vector<char> descs;
    std::vector<BatchUnit> eunits;
    switch (b->storage) {
    case LBM_F32: fill_descs<float, float>(b, descs); edge_units<float, float>(b, eunits); break;
    case LBM_F32_WD_BF16: fill_descs<float, __nv_bfloat16>(b, descs); edge_units<float, __nv_bfloat16>(b, eunits); break;
    case LBM_F32_WD_F16: fill_descs<float, __half>(b, descs); edge_units<float, __half>(b, eunits); break;
    case LBM_F32_LEAPFROG: fill_descs<float, Lf>(b, descs); edge_units<float, Lf>(b, eunits); break;
    default: fill_descs<double, double>(b, descs); edge_units<double, double>(b, eunits); break;
    }
    // D2Q9 lattices with the macroscopic rule on their crack faces: units of
    // 128 columns for the face launch that follows the update
    std::vector<BatchUnit> funits;
    if (b->q == 9)
        for (size_t i = 0; i < b->hs.size(); ++i) {
            const lbm_handle *h = b->hs[i];
            if (!h->cp.macro || h->cp.mode == CRACK_NONE) continue;
            for (int c0 = 0; c0 < h->grid.nx; c0 += 128) funits.push_back(BatchUnit{(int32_t)i, c0, 0, 0});
        }
    std::vector<BatchPiece> pieces;
    std::vector<int32_t> poff;
    if (balanced) {
        lbm_status rc = batch_plan_pieces(b, threads, la, pieces, poff);
        if (rc != LBM_OK) return rc;
    }
    const size_t o_units = align256(descs.size());
    const size_t o_eunits = o_units + align256(units.size() * sizeof(BatchUnit));
    const size_t o_funits = o_eunits + align256(std::max<size_t>(eunits.size(), 1) * sizeof(BatchUnit));
    const size_t o_pieces = o_funits + align256(std::max<size_t>(funits.size(), 1) * sizeof(BatchUnit));
    const size_t o_poff = o_pieces + align256(pieces.size() * sizeof(BatchPiece));
    const size_t need = o_poff + std::max<size_t>(poff.size(), 1) * sizeof(int32_t);
    if (need > b->block_bytes) {
        batch_release_block(b);
        b->block = batch_alloc(b, need);
        if (!b->block) return fail(LBM_ERR_OOM, "device allocation failed");
        b->block_bytes = need;
    }
    b->descs = b->block;
    b->units = reinterpret_cast<BatchUnit *>(static_cast<char *>(b->block) + o_units);
    b->eunits = reinterpret_cast<BatchUnit *>(static_cast<char *>(b->block) + o_eunits);
    b->funits = reinterpret_cast<BatchUnit *>(static_cast<char *>(b->block) + o_funits);
    b->n_funits = (int)funits.size();
    b->pieces = reinterpret_cast<BatchPiece *>(static_cast<char *>(b->block) + o_pieces);
    b->poff = reinterpret_cast<int32_t *>(static_cast<char *>(b->block) + o_poff);
    b->n_units = (int)units.size();
    b->n_eunits = (int)eunits.size();
    b->n_pcta = balanced ? (int)poff.size() - 1 : 0;
    cudaError_t e = cudaMemcpyAsync(b->descs, descs.data(), descs.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !funits.empty())
        e = cudaMemcpyAsync(b->funits, funits.data(), funits.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && balanced && !pieces.empty())
        e = cudaMemcpyAsync(b->pieces, pieces.data(), pieces.size() * sizeof(BatchPiece), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && balanced)
        e = cudaMemcpyAsync(b->poff, poff.data(), poff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->units, units.data(), units.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !eunits.empty())
        e = cudaMemcpyAsync(b->eunits, eunits.data(), eunits.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the batch tables");
    b->graph.reset();
    b->threads = threads;
    b->band_rows = rows;
    b->lookahead = la;
    return LBM_OK;
}

// Shapes chosen by lbm_batch_tune in this process, keyed by the device's SM
// count, the storage and the lattices' sizes and crack bands.
std::mutex g_tune_mu;
struct BatchShape {
    int threads, rows, la;
};
std::map<std::string, BatchShape> g_tune_cache;

std::string batch_key(const lbm_batch *b)
{
    std::vector<std::string> parts;
    for (const lbm_handle *h : b->hs) {
        const int hh = h->cp.mode == CRACK_NONE ? 0 : (h->cp.macro ? 3 : 1);
        parts.push_back(std::to_string(h->grid.nx) + "x" + std::to_string(h->grid.ny) + "/" + std::to_string(h->jc) +
                        "/" + std::to_string(hh) + (h->edge_macro ? "e" : ""));
    }
    std::sort(parts.begin(), parts.end());
    std::string k = std::to_string(b->hs[0]->sms) + "|" + std::to_string(b->storage);
    for (const std::string &p : parts) k += "," + p;
    return k;
}

}  // namespace

namespace lbm {
namespace host {

cudaError_t batch_enqueue(const lbm_batch *b, int par, cudaStream_t s) { return enqueue_batch_step(b, par, s); }

int batch_parity(const lbm_batch *b) { return b->hs[0]->parity; }

lbm_status batch_check(const lbm_batch *b)
{
    const int par0 = b->hs[0]->parity;
    for (lbm_handle *h : b->hs) {
        if (h->sticky != LBM_OK) return fail(h->sticky, "a lattice is in an error state");
        if (h->parity != par0) return fail(LBM_ERR_STATE, "the lattices were stepped apart since the batch was made");
    }
    return LBM_OK;
}

void batch_mark_stepped(lbm_batch *b, int par, int64_t n)
{
    for (lbm_handle *h : b->hs) {
        h->parity = par;
        if (n > 0 && h->cp.mode != CRACK_NONE) h->pending = true;
    }
}

}  // namespace host
}  // namespace lbm

extern "C" {

lbm_status lbm_batch_create(lbm_handle *const *handles, int32_t n, int32_t band_rows, const lbm_allocator *allocator,
                            lbm_batch **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!handles || n < 1) return fail(LBM_ERR_ARG, "need at least one lattice");
    if (band_rows < -1) return fail(LBM_ERR_ARG, "band_rows must be >= 0, or -1 (balanced)");
    for (int i = 0; i < n; ++i) {
        const lbm_handle *h = handles[i];
        if (!h) return fail(LBM_ERR_ARG, "a lattice handle is NULL");
        if (h->sticky != LBM_OK) return fail(h->sticky, "a lattice is in an error state");
        if (h->lat.storage != handles[0]->lat.storage) return fail(LBM_ERR_ARG, "all lattices need the same storage");
        if (h->q != handles[0]->q) return fail(LBM_ERR_ARG, "all lattices need the same velocity set");
        if (h->line != handles[0]->line)
            return fail(LBM_ERR_ARG, "a batch holds cracks along +x or cracks in any direction, not both");
        if (h->stream != handles[0]->stream) return fail(LBM_ERR_ARG, "all lattices need the same stream");
        if (h->parity != handles[0]->parity) return fail(LBM_ERR_STATE, "all lattices need the same number of steps");
        for (int k = 0; k < i; ++k)
            if (handles[k] == h) return fail(LBM_ERR_ARG, "a lattice appears twice");
    }
    lbm_batch *b = new (std::nothrow) lbm_batch;
    if (!b) return fail(LBM_ERR_OOM, "host allocation failed");
    b->hs.assign(handles, handles + n);
    b->storage = handles[0]->lat.storage;
    b->block = nullptr;
    b->block_bytes = 0;
    b->stream = handles[0]->stream;
    b->cap_stream = nullptr;
    b->graph.gen = -1;
    b->q = handles[0]->q;
    b->line = handles[0]->line;
    b->funits = nullptr;
    b->n_funits = 0;
    b->pieces = nullptr;
    b->poff = nullptr;
    b->n_pcta = 0;
    b->threads = kThreads;
    b->band_rows = 16;
    b->lookahead = 1;
    b->chained = false;
    b->persistent = false;
    b->budget = (long long)1 << 31;
    b->bar = nullptr;
    b->err = nullptr;
    b->custom_alloc = allocator && allocator->alloc && allocator->release;
    if (b->custom_alloc) b->alloc = *allocator;
    b->owns = false;
    auto bail = [&](lbm_status rc) {
        batch_release_block(b);
        batch_free(b, b->bar);
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        delete b;
        return rc;
    };
    b->bar = static_cast<GridBarrier *>(batch_alloc(b, 256));
    if (!b->bar) return bail(fail(LBM_ERR_OOM, "device allocation failed"));
    b->err = reinterpret_cast<uint32_t *>(static_cast<char *>(static_cast<void *>(b->bar)) + 128);
    {
        cudaError_t e = cudaMemsetAsync(b->bar, 0, 256, b->stream);
        if (e != cudaSuccess) return bail(cuda_fail(e, "clearing the batch barrier"));
    }
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaStreamSynchronize(handles[i]->stream);
        if (e != cudaSuccess) return bail(cuda_fail(e, "synchronising a lattice"));
    }
    // bands of band_rows rows (default 16), CTAs of 128 threads: a batch has
    // many CTAs, no need to fit one wave; lbm_batch_tune picks a better shape
    lbm_status rc = batch_build(b, kThreads, band_rows != 0 ? band_rows : 16, 1);
    if (rc != LBM_OK) return bail(rc);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "creating the capture stream"));
    *out = b;
    clear_error();
    return LBM_OK;
}

lbm_status lbm_batch_set_shape(lbm_batch *b, int32_t threads, int32_t band_rows)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    lbm_status rc = batch_check(b);
    if (rc != LBM_OK) return rc;
    for (lbm_handle *h : b->hs) LBM_CUDA(cudaStreamSynchronize(h->stream));
    rc = batch_build(b, threads, band_rows, b->lookahead);
    if (rc == LBM_OK) clear_error();
    return rc;
}

lbm_status lbm_batch_set_lookahead(lbm_batch *b, int32_t rows)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    if (rows != 1 && rows != 2) return fail(LBM_ERR_ARG, "lookahead must be 1 or 2 rows");
    lbm_status rc = batch_check(b);
    if (rc != LBM_OK) return rc;
    for (lbm_handle *h : b->hs) LBM_CUDA(cudaStreamSynchronize(h->stream));
    rc = batch_build(b, b->threads, b->band_rows, rows);
    if (rc == LBM_OK) clear_error();
    return rc;
}

lbm_status lbm_batch_set_chained(lbm_batch *b, int32_t enable)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    lbm_status rc = batch_check(b);
    if (rc != LBM_OK) return rc;
    for (lbm_handle *h : b->hs) LBM_CUDA(cudaStreamSynchronize(h->stream));
    b->chained = enable != 0;
    b->graph.reset();
    clear_error();
    return LBM_OK;
}

lbm_status lbm_batch_get_lookahead(const lbm_batch *b, int32_t *rows)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    if (rows) *rows = b->lookahead;
    return LBM_OK;
}

lbm_status lbm_batch_get_shape(const lbm_batch *b, int32_t *threads, int32_t *band_rows)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    if (threads) *threads = b->threads;
    if (band_rows) *band_rows = b->band_rows;
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, int32_t *threads, int32_t *band_rows,
                          double *us_per_step, int32_t *from_cache)
{
    lbm::NvtxRange nvtx_("lbm_batch_tune");
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    if (trial_steps < 2 || trial_steps > 1024) return fail(LBM_ERR_ARG, "trial_steps must be in [2, 1024]");
    lbm_status rc = batch_check(b);
    if (rc != LBM_OK) return rc;
    const std::string key = batch_key(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            for (lbm_handle *h : b->hs) LBM_CUDA(cudaStreamSynchronize(h->stream));
            rc = batch_build(b, it->second.threads, it->second.rows, it->second.la);
            if (rc != LBM_OK) return rc;
            if (threads) *threads = b->threads;
            if (band_rows) *band_rows = b->band_rows;
            if (us_per_step) *us_per_step = 0.0;
            if (from_cache) *from_cache = 1;
            clear_error();
            return LBM_OK;
        }
    }
    // the trials advance the lattices: keep every lattice's device block and
    // host step state, and put them back afterwards
    for (lbm_handle *h : b->hs) {
        rc = finalize(h);
        if (rc != LBM_OK) return rc;
        LBM_CUDA(cudaStreamSynchronize(h->stream));
    }
    size_t total = 0;
    std::vector<size_t> off;
    for (lbm_handle *h : b->hs) {
        off.push_back(total);
        total = align256(total + h->block_bytes);
    }
    void *snap = batch_alloc(b, std::max<size_t>(total, 256));
    if (!snap) return fail(LBM_ERR_OOM, "device allocation failed (state snapshot for the trials)");
    std::vector<int> par0;
    std::vector<bool> pend0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto done = [&](lbm_status r) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamSynchronize(b->stream);
        batch_free(b, snap);
        return r;
    };
    for (size_t i = 0; i < b->hs.size(); ++i) {
        lbm_handle *h = b->hs[i];
        par0.push_back(h->parity);
        pend0.push_back(h->pending);
        cudaError_t e = cudaMemcpyAsync(static_cast<char *>(snap) + off[i], h->block, h->block_bytes,
                                        cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return done(cuda_fail(e, "saving the lattices' state"));
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return done(fail(LBM_ERR_CUDA, "creating timing events"));
    const int shapes_t[3] = {32, 64, kThreads};
    const int shapes_r[7] = {-1, 0, 8, 16, 32, 64, -2};   // -1: balanced; 0: one wave; -2: tapered
    int best_t = b->threads, best_r = b->band_rows, best_la = b->lookahead;
    double best = 1e300;
    int par = b->hs[0]->parity;
    // a D2Q9 batch: CTAs of 128 threads, a lookahead of one row, bands only;
    // a batch of cracks in any direction: its lattices' fixed grids, one shape
    const bool d9 = b->q == 9 || b->line;
    for (int la = 1; la <= (d9 ? 1 : 2); ++la)
        for (int ti = d9 ? 2 : 0; ti < 3; ++ti)
            for (int ri = d9 ? 1 : 0; ri < (b->line ? 2 : 7); ++ri) {
                rc = batch_build(b, shapes_t[ti], shapes_r[ri], la);
                if (rc != LBM_OK) return done(rc);
                double t_min = 1e300;
                for (int rep = 0; rep < 3; ++rep) {
                    cudaError_t e = cudaEventRecord(e0, b->stream);
                    for (int q = 0; q < trial_steps && e == cudaSuccess; ++q) {
                        e = enqueue_batch_step(b, par, b->stream);
                        par ^= 1;
                    }
                    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) return done(cuda_fail(e, "timing a batch shape"));
                    if (rep > 0) t_min = std::min(t_min, (double)ms);   // the first repetition warms up
                }
                if (t_min < best) {
                    best = t_min;
                    best_t = shapes_t[ti];
                    best_r = shapes_r[ri];
                    best_la = la;
                }
            }
    for (size_t i = 0; i < b->hs.size(); ++i) {
        lbm_handle *h = b->hs[i];
        cudaError_t e = cudaMemcpyAsync(h->block, static_cast<char *>(snap) + off[i], h->block_bytes,
                                        cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return done(cuda_fail(e, "restoring the lattices' state"));
        h->parity = par0[i];
        h->pending = pend0[i];
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return done(cuda_fail(e, "restoring the lattices' state"));
    // the restored blocks hold the unit tables of the shape in force at the
    // snapshot: partition again for the chosen shape
    rc = batch_build(b, best_t, best_r, best_la);
    if (rc != LBM_OK) return done(rc);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = BatchShape{best_t, best_r, best_la};
    }
    if (threads) *threads = best_t;
    if (band_rows) *band_rows = best_r;
    if (us_per_step) *us_per_step = best * 1e3 / trial_steps;
    if (from_cache) *from_cache = 0;
    clear_error();
    return done(LBM_OK);
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t n)
{
    lbm::NvtxRange nvtx_("lbm_batch_step");
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
    const int par0 = b->hs[0]->parity;
    for (lbm_handle *h : b->hs) {
        if (h->sticky != LBM_OK) return fail(h->sticky, "a lattice is in an error state");
        if (h->parity != par0) return fail(LBM_ERR_STATE, "the lattices were stepped apart since the batch was made");
    }
    int par = par0;
    int64_t left = n;
    if (b->persistent && n > 0) {
        LBM_CUDA(enqueue_batch_persistent(b, par, n, b->stream));
        par ^= (int)(n & 1);
        left = 0;
    }
    if (left > 0) {
        // runs of steps replay graphs of 64, 32, ..., 2 batched steps
        const lbm_status rc = run_chunks(b->graph, 0, b->stream, b->cap_stream, left, par,
                                         [&](int p, cudaStream_t s) { return enqueue_batch_step(b, p, s); });
        if (rc != LBM_OK) return rc;
    }
    for (lbm_handle *h : b->hs) {
        h->parity = par;
        if (n > 0 && h->cp.mode != CRACK_NONE) h->pending = true;
    }
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch *b, int32_t *n_lattices, int32_t *ctas)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    if (n_lattices) *n_lattices = (int32_t)b->hs.size();
    if (ctas) *ctas = b->n_pcta > 0 ? b->n_pcta : b->n_units;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    b->graph.reset();
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    batch_release_block(b);
    batch_free(b, b->bar);
    if (b->owns)
        for (lbm_handle *h : b->hs) lbm_destroy(h);
    delete b;
}

lbm_status lbm_create_batch(int32_t n, const lbm_grid *grids, const lbm_lattice *lattices, const lbm_material *materials,
                            const lbm_crack *cracks, const lbm_loading *const *loads, const int32_t *n_loads,
                            void *stream, const lbm_allocator *allocator, int32_t band_rows, lbm_batch **out)
{
    lbm::NvtxRange nvtx_("lbm_create_batch");
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !grids || !lattices || !materials) return fail(LBM_ERR_ARG, "need n >= 1 and the grid, lattice and material arrays");
    if ((loads == nullptr) != (n_loads == nullptr)) return fail(LBM_ERR_ARG, "loads and n_loads come together");
    std::vector<lbm_handle *> hs;
    hs.reserve((size_t)n);
    auto drop = [&](lbm_status rc) {
        const std::string msg = last_error();
        for (lbm_handle *h : hs) lbm_destroy(h);
        return fail(rc, "lattice " + std::to_string(hs.size()) + ": " + msg);
    };
    for (int32_t i = 0; i < n; ++i) {
        lbm_handle *h = nullptr;
        lbm_status rc = lbm_create(grids + i, lattices + i, materials + i, cracks ? cracks + i : nullptr,
                                   loads ? loads[i] : nullptr, n_loads ? n_loads[i] : 0, stream, allocator, &h);
        if (rc != LBM_OK) return drop(rc);
        hs.push_back(h);
    }
    lbm_batch *b = nullptr;
    lbm_status rc = lbm_batch_create(hs.data(), n, band_rows, allocator, &b);
    if (rc != LBM_OK) {
        const std::string msg = last_error();
        for (lbm_handle *h : hs) lbm_destroy(h);
        return fail(rc, msg);
    }
    b->owns = true;
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_member(const lbm_batch *b, int32_t i, lbm_handle **h)
{
    if (!b || !h) return fail(LBM_ERR_ARG, "batch or h is NULL");
    if (i < 0 || i >= (int32_t)b->hs.size()) return fail(LBM_ERR_ARG, "member index out of range");
    *h = b->hs[(size_t)i];
    return LBM_OK;
}

lbm_status lbm_batch_set_persistent(lbm_batch *b, int32_t enable, int64_t budget_cycles)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    if (budget_cycles < 0 || budget_cycles > ((int64_t)1 << 40)) return fail(LBM_ERR_ARG, "budget out of range");
    if (enable && (b->q == 9 || b->line))
        return fail(LBM_ERR_ARG, "the persistent batched step is built for D2Q5 cracks along +x only");
    b->persistent = enable != 0;
    b->budget = budget_cycles > 0 ? (long long)budget_cycles : (long long)1 << 31;
    clear_error();
    return LBM_OK;
}

lbm_status lbm_barrier_probe(int32_t ctas, int32_t expected, int64_t budget_cycles, void *stream)
{
    if (ctas < 1 || ctas > 64 || expected < 1 || expected > 64) return fail(LBM_ERR_ARG, "ctas and expected in [1, 64]");
    if (budget_cycles < 1000 || budget_cycles > ((int64_t)1 << 34)) return fail(LBM_ERR_ARG, "budget out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *mem = nullptr;
    LBM_CUDA(cudaMalloc(&mem, 256));
    GridBarrier *bar = static_cast<GridBarrier *>(mem);
    uint32_t *err = reinterpret_cast<uint32_t *>(static_cast<char *>(mem) + 128);
    uint32_t host_err = 0;
    cudaError_t e = cudaMemsetAsync(mem, 0, 256, s);
    if (e == cudaSuccess) e = launch_barrier_probe(bar, ctas, expected, (long long)budget_cycles, err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, err, sizeof host_err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_fail(e, "running the barrier probe");
    if (host_err & ERR_TIMEOUT) return fail(LBM_ERR_TIMEOUT, "the bounded wait at the grid barrier gave up");
    clear_error();
    return LBM_OK;
}

const char *lbm_last_error(void) { return last_error(); }

}  // extern "C"
