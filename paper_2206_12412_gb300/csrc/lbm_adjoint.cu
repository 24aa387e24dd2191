// lbm_adjoint.cu -- CUDA kernels (sm_103a) of the adjoint of the time step
// (arXiv 2206.12412, Sec. 3 and 3.1) under a recorded cut schedule.
//
// With the crack's cut schedule held fixed, one time step is affine in the
// state (w, wdot):
//     v^ = wdot + g (L_n w + b_n),   w^ = w + dt v^,
// L_n the five-point stencil with bounce-back on severed links and free
// edges, anti-bounce-back on Dirichlet edges (diagonal -1) and periodic wrap,
// b_n = 2 w*(t_n) on sites next to a Dirichlet edge; then, with macroscopic
// crack faces, at every boundary point x_B of a severed column (rows jc-1,
// jc) w'(x_B) = 1.5 w^(x_I) - 0.5 w^(x_II) (x_I, x_II one and two rows further
// from the crack) and wdot'(x_B) = (w'(x_B) - w(x_B)) / dt; elsewhere w' = w^,
// wdot' = v^.  L_n is symmetric, so its transpose is the same stencil.
//
// Transposing the step: with (alpha, beta) = (dL/dw, dL/dwdot) after the step
// and m~ = beta + dt alpha, the adjoint of v^ is mu and
//     dL/dw = a + g L_n mu,     dL/dwdot = mu,
// where a = alpha and mu = m~ away from the crack faces, and at the boundary
// points of the columns severed in the step
//     mu_B = 0,                a_B = alpha_B - m~_B / dt,
//     mu_I = m~_I + 1.5 m~_B,  a_I = alpha_I + 1.5 m~_B / dt,
//     mu_II = m~_II - 0.5 m~_B, a_II = alpha_II - 0.5 m~_B / dt.
// The kernel keeps the pair (m, a) = (mu, a) of the next transposed step in
// the layout of (w, wdot): m in ping-pong planes with pads, a in place.  One
// kernel step computes alpha = a + g L_n m and m~ = m + dt alpha -- the
// forward update with zero Dirichlet values -- adds the sensor sources of
// the state (dL/dw(x_s) = 2 r_s into alpha, 2 r_s dt into m~), and applies
// the correction above for the columns severed in the previous forward step,
// which is local to each column of the crack sub-bands.  It moves the same
// 16 bytes per site as the forward step and needs no forward state: only the
// recorded cut schedule (the last severed column of each step) and the
// recorded sensor misfits.  dL/dw*_e(t_n) = 2 g times the sum of m over the
// sites next to edge e (per-CTA partial sums in FP64, added in a fixed order
// by a second kernel).
#include "lbm_internal.cuh"
#include "lbm_rows.cuh"

namespace lbm {

// Bits k (0 <= k < N) of the columns x0 + k in [lo, hi].
template <int N>
__device__ __forceinline__ uint32_t col_bits(int x0, int lo, int hi)
{
    uint32_t b = 0u;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (x0 + k >= lo && x0 + k <= hi) b |= 1u << k;
    return b;
}

// The sensor sources of state n that fall in one CTA: the first kMaxSrc of
// its list staged in shared memory (site and value 2 r), any further ones
// read from the global list.
constexpr int kMaxSrc = 64;

template <typename T> struct SrcTab {
    const int32_t *sj, *si;   // shared memory, n_s entries
    const T *sv;
    int n_s;
    int lo_g, hi_g;           // entries of the global list that were not staged
    int64_t srow;             // misfit row of state n
};

// Sources on row j of this thread's columns: each sensor there adds 2 r to
// alpha and 2 r dt to m.
template <typename T, int N>
__device__ __forceinline__ void add_sources(const AdjArgs<T> &a, const SrcTab<T> &S, int x0, int j, Row<T, N> &anew,
                                            Row<T, N> &mnew)
{
    for (int q = 0; q < S.n_s; ++q) {
        if (S.sj[q] != j) continue;
        const int di = S.si[q] - x0;
        if (di < 0 || di >= N) continue;
        const T v = S.sv[q];
#pragma unroll
        for (int kk = 0; kk < N; ++kk)
            if (kk == di) {
                anew.v[kk] += v;
                mnew.v[kk] += a.dt * v;
            }
    }
    const int64_t srow = S.srow;
    for (int q = S.lo_g; q < S.hi_g; ++q) {
        const int k = a.s_ent[q];
        if (a.s_j[k] != j) continue;
        const int di = a.s_i[k] - x0;
        if (di < 0 || di >= N) continue;
        const T v = (T)(2.0 * a.resid[srow * a.ns + k]);
#pragma unroll
        for (int kk = 0; kk < N; ++kk)
            if (kk == di) {
                anew.v[kk] += v;
                mnew.v[kk] += a.dt * v;
            }
    }
}

// Sums of m (the input plane) along the Dirichlet edges that this CTA
// touches, over its own sites, in FP64: the thread's columns of row 0 /
// ny - 1, and rows j0 .. j1-1 of column 0 / nx - 1.  Read back after the
// march (the input plane is not written during the step), so that no
// accumulator lives through the row loop.
template <typename T>
__device__ __forceinline__ void edge_sums(const AdjArgs<T> &a, int x0, int j0, int j1, bool on_t, bool on_b, bool on_l,
                                          bool on_r, double (&es)[4])
{
    constexpr int N = Vec<T>::N;
    const int64_t P = a.pitch;
    const int nx = a.nx;
#pragma unroll
    for (int e = 0; e < 4; ++e) es[e] = 0.0;
    if (on_t || on_b) {
        const T *row = a.w_in + (on_t ? (int64_t)(a.ny - 1) * P : 0) + x0;
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (x0 + k < nx) s += (double)row[k];
        es[on_t ? TOP : BOTTOM] = s;
    }
    if (on_l && x0 == 0)
        for (int j = j0; j < j1; ++j) es[LEFT] += (double)a.w_in[(int64_t)j * P];
    if (on_r && x0 <= nx - 1 && nx - 1 < x0 + N)
        for (int j = j0; j < j1; ++j) es[RIGHT] += (double)a.w_in[(int64_t)j * P + nx - 1];
}

// The bulk rows: the forward march with zero Dirichlet values and the
// sources (SRC).
template <typename T, bool EDGE, bool SRC>
__device__ __forceinline__ void adj_march(const AdjArgs<T> &a, int cb, int j0, int j1, const SrcTab<T> &S, T &acc)
{
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int x0 = (cb * kThreads + threadIdx.x) * N;
    const int64_t P = a.pitch;
    const T *mip = a.w_in + x0;
    T *mout = a.w_out + x0;
    T *ap = a.wd + x0;
    R mb, mc, ma, av;
    ldg_row(mip + (int64_t)(j0 - 1) * P, mb);
    ldg_row(mip + (int64_t)j0 * P, mc);
    ldg_row(mip + (int64_t)(j0 + 1) * P, ma);
    ld_row(ap + (int64_t)j0 * P, av);
    T hl = (T)0, hr = (T)0;
    if (lane == 0) hl = mip[(int64_t)j0 * P - 1];
    if (lane == 31) hr = mip[(int64_t)j0 * P + N];
    const T g = a.g, dt = a.dt;
    EdgeValues<T> E;
#pragma unroll
    for (int e = 0; e < 4; ++e) E.two_ws[e] = (T)0;
    for (int j = j0; j < j1; ++j) {
        R mn, an;
        T hln = (T)0, hrn = (T)0;
        const bool more = j + 1 < j1;
        if (more) {
            ldg_row(mip + (int64_t)(j + 2) * P, mn);
            ld_row(ap + (int64_t)(j + 1) * P, an);
            if (lane == 0) hln = mip[(int64_t)(j + 1) * P - 1];
            if (lane == 31) hrn = mip[(int64_t)(j + 1) * P + N];
        }
        T left0 = __shfl_up_sync(kFull, mc.v[N - 1], 1);
        T rightN = __shfl_down_sync(kFull, mc.v[0], 1);
        if (lane == 0) left0 = hl;
        if (lane == 31) rightN = hr;
        R mnew, anew;
        if (EDGE) {
            row_update(a, E, x0, j, mc, ma, mb, av, left0, rightN, 0u, 0u, mnew, anew);
            if (SRC) add_sources<T, N>(a, S, x0, j, anew, mnew);
            if (x0 < a.nx) {
                store_row(a, x0, j, mnew, anew, acc);
                write_pads(a, x0, j, mnew);
            }
        } else {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const T ml = k == 0 ? left0 : mc.v[k - 1];
                const T mr = k == N - 1 ? rightN : mc.v[k + 1];
                const T lap = ((ma.v[k] + mb.v[k]) + (ml + mr)) - (T)4 * mc.v[k];
                anew.v[k] = av.v[k] + g * lap;
                mnew.v[k] = mc.v[k] + dt * anew.v[k];
            }
            if (SRC) add_sources<T, N>(a, S, x0, j, anew, mnew);
            stg_row(mout + (int64_t)j * P, mnew);
            stg_row(ap + (int64_t)j * P, anew);
            acc += mnew.v[0];
        }
        mb = mc;
        mc = ma;
        if (more) {
            ma = mn;
            av = an;
            hl = hln;
            hr = hrn;
        }
    }
}

// A crack sub-band of HH rows (rows jc-HH .. jc-1 or jc .. jc+HH-1): the
// stencil with the severed links of step n (columns if_n .. il_n), the
// sources, then the crack-face correction for the columns severed in step
// n - 1 (if_p .. il_p), all from registers.  Out of line (its register
// demand would otherwise be the whole kernel's), with the arguments in shared
// memory; returns the finiteness probe.
template <typename T, int HH>
__device__ __noinline__ T adj_crack_rows(const AdjArgs<T> *sa, int cb, int j0, int if_n, int il_n, int if_p, int il_p,
                                         const int32_t *ssj,
                                         const int32_t *ssi, const T *ssv, int n_s, int lo_g, int hi_g, int64_t srow)
{
    const AdjArgs<T> &a = *sa;
    SrcTab<T> S;
    S.sj = ssj;
    S.si = ssi;
    S.sv = ssv;
    S.n_s = n_s;
    S.lo_g = lo_g;
    S.hi_g = hi_g;
    S.srow = srow;
    T acc = (T)0;
    constexpr int N = Vec<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int x0 = (cb * kThreads + threadIdx.x) * N;
    const int jc = a.jc;
    const int64_t P = a.pitch;
    const T *mip = a.w_in + x0;
    const bool below = j0 + HH == jc;
    R m[HH + 2], av[HH];
    T hl[HH], hr[HH];
#pragma unroll
    for (int q = 0; q < HH + 2; ++q) ldg_row(mip + (int64_t)(j0 - 1 + q) * P, m[q]);
#pragma unroll
    for (int q = 0; q < HH; ++q) {
        ld_row(a.wd + x0 + (int64_t)(j0 + q) * P, av[q]);
        hl[q] = lane == 0 ? mip[(int64_t)(j0 + q) * P - 1] : (T)0;
        hr[q] = lane == 31 ? mip[(int64_t)(j0 + q) * P + N] : (T)0;
    }
    EdgeValues<T> E;
#pragma unroll
    for (int e = 0; e < 4; ++e) E.two_ws[e] = (T)0;
    const uint32_t cut_n = col_bits<N>(x0, if_n, il_n);
    const uint32_t cut_p = col_bits<N>(x0, if_p, il_p);
    R o[HH], od[HH];
#pragma unroll
    for (int q = 0; q < HH; ++q) {
        const int j = j0 + q;
        T left0 = __shfl_up_sync(kFull, m[q + 1].v[N - 1], 1);
        T rightN = __shfl_down_sync(kFull, m[q + 1].v[0], 1);
        if (lane == 0) left0 = hl[q];
        if (lane == 31) rightN = hr[q];
        const uint32_t cut_up = (below && j == jc - 1) ? cut_n : 0u;
        const uint32_t cut_dn = (!below && j == jc) ? cut_n : 0u;
        row_update(a, E, x0, j, m[q + 1], m[q + 2], m[q], av[q], left0, rightN, cut_up, cut_dn, o[q], od[q]);
        add_sources<T, N>(a, S, x0, j, od[q], o[q]);
    }
    if (HH >= 3 && a.macro && cut_p) {
        const int qb = below ? HH - 1 : 0, qi = below ? HH - 2 : 1, qii = below ? HH - 3 : 2;
        const T inv_dt = (T)1 / a.dt;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if ((cut_p >> k) & 1u) {
                const T mB = o[qb].v[k];
                od[qb].v[k] -= mB * inv_dt;
                o[qb].v[k] = (T)0;
                od[qi].v[k] += (T)1.5 * mB * inv_dt;
                o[qi].v[k] += (T)1.5 * mB;
                od[qii].v[k] -= (T)0.5 * mB * inv_dt;
                o[qii].v[k] -= (T)0.5 * mB;
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

template <typename T>
__device__ __forceinline__ void adjoint_cta(const AdjArgs<T> &a, int cb, int band, double *sred, AdjArgs<T> *sa,
                                            int32_t *ssj, int32_t *ssi, T *ssv)
{
    const unsigned kFull = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t n = *a.cnt_in;
    if (cb == 0 && band == 0 && tid == 0) *a.cnt_out = n - 1;
    n = n < 0 ? 0 : (n > a.n_steps ? a.n_steps : n);   // the host launches exactly n_steps + 1 steps
    const Unit U = a.units[band];
    const int j0 = U.j0, j1 = U.j1;
    int lo = 0, hi = 0;
    int64_t srow = 0;
    if (n >= 1 && a.ns > 0) {
        const int u = band * a.ncb + cb;
        lo = a.s_off[u];
        hi = a.s_off[u + 1];
        srow = (n - 1) % a.ring;
    }
    // stage this CTA's sources (the count is the same for all its threads)
    const int n_s = min(hi - lo, kMaxSrc);
    if (n_s > 0) {
        for (int q = tid; q < n_s; q += kThreads) {
            const int k = a.s_ent[lo + q];
            ssj[q] = a.s_j[k];
            ssi[q] = a.s_i[k];
            ssv[q] = (T)(2.0 * a.resid[srow * a.ns + k]);
        }
        __syncthreads();
    }
    SrcTab<T> S;
    S.sj = ssj;
    S.si = ssi;
    S.sv = ssv;
    S.n_s = n_s;
    S.lo_g = lo + n_s;
    S.hi_g = hi;
    S.srow = srow;
    T acc;
    if (a.crack_band >= 0 && (band == a.crack_band || band == a.crack_band + 1)) {
        const int64_t nn = n < a.n_steps ? n : a.n_steps - 1;
        const int if_n = a.i_first[nn], il_n = a.i_last[nn];
        const int if_p = n >= 1 ? a.i_first[n - 1] : 1, il_p = n >= 1 ? a.i_last[n - 1] : 0;   // none before step 0
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&a);
        uint32_t *dst = reinterpret_cast<uint32_t *>(sa);
        for (int q = tid; q < (int)(sizeof(AdjArgs<T>) / 4); q += kThreads) dst[q] = src[q];
        __syncthreads();
        acc = a.macro ? adj_crack_rows<T, 3>(sa, cb, j0, if_n, il_n, if_p, il_p, ssj, ssi, ssv, n_s, lo + n_s, hi, srow)
                      : adj_crack_rows<T, 1>(sa, cb, j0, if_n, il_n, if_p, il_p, ssj, ssi, ssv, n_s, lo + n_s, hi, srow);
    } else {
        acc = (T)0;
        const bool edge = (cb == 0) | (cb == a.ncb - 1) | (j0 == 0) | (j1 == a.ny);
        const bool src = lo < hi;
        if (edge) {
            if (src) adj_march<T, true, true>(a, cb, j0, j1, S, acc);
            else adj_march<T, true, false>(a, cb, j0, j1, S, acc);
        } else {
            if (src) adj_march<T, false, true>(a, cb, j0, j1, S, acc);
            else adj_march<T, false, false>(a, cb, j0, j1, S, acc);
        }
    }
    if (__any_sync(kFull, !isfinite(acc)) && lane == 0) atomicOr(a.err, (uint32_t)ERR_NONFINITE);
    // per-CTA sums of m along the Dirichlet edges this CTA touches
    const bool on_t = j1 == a.ny && a.edge[TOP] == EDGE_DIRICHLET;
    const bool on_b = j0 == 0 && a.edge[BOTTOM] == EDGE_DIRICHLET;
    const bool on_l = cb == 0 && a.edge[LEFT] == EDGE_DIRICHLET;
    const bool on_r = cb == a.ncb - 1 && a.edge[RIGHT] == EDGE_DIRICHLET;
    if ((on_t | on_b | on_l | on_r) && n < a.n_steps) {
        double es[4];
        edge_sums<T>(a, (cb * kThreads + tid) * Vec<T>::N, j0, j1, on_t, on_b, on_l, on_r, es);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            double v = es[e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0) sred[warp * 4 + e] = v;
        }
        __syncthreads();
        if (tid == 0) {
            double s[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                s[e] = 0.0;
                for (int w = 0; w < kThreads / 32; ++w) s[e] += sred[w * 4 + e];
            }
            double *pn = a.part + (size_t)n * 4 * (size_t)a.slots;
            if (on_t) pn[TOP * a.slots + cb] = s[TOP];
            if (on_b) pn[BOTTOM * a.slots + cb] = s[BOTTOM];
            if (on_l) pn[LEFT * a.slots + band] = s[LEFT];
            if (on_r) pn[RIGHT * a.slots + band] = s[RIGHT];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : kMinBlocks - 2) adjoint_kernel(const AdjArgs<T> a)
{
    __shared__ double sred[4 * (kThreads / 32)];
    __shared__ __align__(16) AdjArgs<T> sa;
    __shared__ int32_t ssj[kMaxSrc], ssi[kMaxSrc];
    __shared__ T ssv[kMaxSrc];
    adjoint_cta<T>(a, blockIdx.x, blockIdx.y, sred, &sa, ssj, ssi, ssv);
}

template <typename T> const void *adjoint_kernel_ptr()
{
    return reinterpret_cast<const void *>(&adjoint_kernel<T>);
}

template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T> &a, int bands, cudaStream_t s)
{
    adjoint_kernel<T><<<dim3((unsigned)a.ncb, (unsigned)bands), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ reductions

// L = sum_k acc[k], in sensor order (one thread).
__global__ void loss_sum_kernel(const double *acc, int ns, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < ns; ++k) s += acc[k];
        *out = s;
    }
}

cudaError_t launch_loss_sum(const double *acc, int ns, double *out, cudaStream_t s)
{
    loss_sum_kernel<<<1, 32, 0, s>>>(acc, ns, out);
    return cudaGetLastError();
}

// grad[e][n] = 2 g sum_slot part[n][e][slot] for Dirichlet edges (bit e of
// dir_mask), 0 otherwise; slots summed in order.
__global__ void grad_sum_kernel(const double *part, int64_t T, int slots, int dir_mask, double g, double *grad)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * T) return;
    const int e = (int)(t / T);
    const int64_t n = t % T;
    double s = 0.0;
    if ((dir_mask >> e) & 1) {
        const double *p = part + ((size_t)n * 4 + (size_t)e) * (size_t)slots;
        for (int q = 0; q < slots; ++q) s += p[q];
    }
    grad[t] = 2.0 * g * s;
}

cudaError_t launch_grad_sum(const double *part, int64_t T, int slots, int dir_mask, double g, double *grad,
                            cudaStream_t s)
{
    const int64_t n = 4 * T;
    grad_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, T, slots, dir_mask, g, grad);
    return cudaGetLastError();
}

// dL/dw0 = a, dL/dwdot0 = m - dt a, as dense ny x nx arrays.
template <typename T>
__global__ void adjoint_out_kernel(const T *a, const T *m, int64_t P, int nx, int ny, T dt, T *dw, T *dwd)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nx * ny) return;
    const int j = (int)(t / nx), i = (int)(t % nx);
    const T av = a[(int64_t)j * P + i];
    dw[t] = av;
    dwd[t] = m[(int64_t)j * P + i] - dt * av;
}

template <typename T>
cudaError_t launch_adjoint_out(const T *a, const T *m, int64_t pitch, int nx, int ny, T dt, T *dw, T *dwd, cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny;
    adjoint_out_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, m, pitch, nx, ny, dt, dw, dwd);
    return cudaGetLastError();
}

template const void *adjoint_kernel_ptr<float>();
template const void *adjoint_kernel_ptr<double>();
template cudaError_t launch_adjoint<float>(const AdjArgs<float> &, int, cudaStream_t);
template cudaError_t launch_adjoint<double>(const AdjArgs<double> &, int, cudaStream_t);
template cudaError_t launch_adjoint_out<float>(const float *, const float *, int64_t, int, int, float, float *, float *,
                                               cudaStream_t);
template cudaError_t launch_adjoint_out<double>(const double *, const double *, int64_t, int, int, double, double *,
                                                double *, cudaStream_t);

}  // namespace lbm
