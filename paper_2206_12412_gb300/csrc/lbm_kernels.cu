// lbm_kernels.cu -- CUDA kernels (sm_103a) of one lattice Boltzmann time step
// for antiplane shear with dynamic mode III cracks (arXiv 2206.12412).
//
// Moment form.  With tau = dt (Sec. 3) the BGK collision sets every
// distribution to its equilibrium, f*^k = g w (k = 1..4), f*^0 = wdot - 4 g w
// (eq. f-eq, read so that sum_a f_eq^a = wdot; g = c_s^2 dt / dh^2), so the
// pair (w, wdot) is the whole state.  Streaming f*^k from the four neighbours
// and summing (eq. distrib-macro) gives
//     wdot' = wdot + g * (w_N + w_S + w_E + w_W - 4 w),     w' = w + dt wdot'
// (eq. integration), where a missing link contributes the value its boundary
// rule streams back: bounce-back f*^opp(x) = g w(x) (free edge, severed crack
// link), anti-bounce-back -f*^opp(x) + 2 g w* = g (2 w* - w(x)) (Dirichlet
// edge, Sec. 3.1), or the periodic image.  The bulk kernel therefore moves
// exactly 16 bytes per site in FP32 (read w, wdot; write w, wdot).
#include "lbm_internal.cuh"

namespace lbm {

template <typename T> struct VecOf;
template <> struct VecOf<float> { typedef float4 V; static constexpr int N = 4; };
template <> struct VecOf<double> { typedef double2 V; static constexpr int N = 2; };

template <typename T, int N> struct Row { T v[N]; };

__device__ __forceinline__ void ld_row(const float *p, Row<float, 4> &r)
{
    float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
}
__device__ __forceinline__ void ld_row(const double *p, Row<double, 2> &r)
{
    double2 q = __ldg(reinterpret_cast<const double2 *>(p));
    r.v[0] = q.x; r.v[1] = q.y;
}
// wdot is updated in place: plain (coherent) loads.
__device__ __forceinline__ void ld_row_rw(const float *p, Row<float, 4> &r)
{
    float4 q = *reinterpret_cast<const float4 *>(p);
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
}
__device__ __forceinline__ void ld_row_rw(const double *p, Row<double, 2> &r)
{
    double2 q = *reinterpret_cast<const double2 *>(p);
    r.v[0] = q.x; r.v[1] = q.y;
}
__device__ __forceinline__ void st_row(float *p, const Row<float, 4> &r)
{
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
}
__device__ __forceinline__ void st_row(double *p, const Row<double, 2> &r)
{
    *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
}

// Value streamed across a missing outer-edge link.
template <typename T>
__device__ __forceinline__ T edge_value(int kind, T wstar, T wc, T raw)
{
    if (kind == EDGE_FREE) return wc;                        // bounce-back
    if (kind == EDGE_DIRICHLET) return (T)2 * wstar - wc;    // anti-bounce-back
    return raw;                                              // periodic image in the pad
}

// ---------------------------------------------------------------- bulk step
//
// Thread mapping: a thread owns N consecutive columns (one 16-byte vector) and
// marches over `rows` consecutive rows, keeping rows j-1, j, j+1 of w in
// registers, so each w value is loaded from memory once per step (plus one
// halo row per strip end).  East/west neighbours come from the adjacent lanes
// by warp shuffles; lanes 0 and 31 load the one halo column they need.  The
// next row's loads are issued before the current row is computed.
template <typename T>
__global__ void __launch_bounds__(kBulkThreads) bulk_kernel(const BulkArgs<T> a)
{
    constexpr int N = VecOf<T>::N;
    typedef Row<T, N> R;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * kBulkThreads + threadIdx.x) * N;
    const int j0 = blockIdx.y * a.rows;
    const int j1 = min(j0 + a.rows, a.ny);
    const int64_t P = a.pitch;
    const int nx = a.nx, ny = a.ny;
    if (j0 >= ny) return;  // uniform per block

    T ws[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) ws[e] = (T)a.st->wstar[e];

    const bool act = x0 < nx;
    const bool col_edge = (x0 == 0) | (x0 + N >= nx);
    const T *win = a.w_in + x0;
    T *wout = a.w_out + x0;
    T *wdp = a.wd + x0;
    const int wi = x0 >> 5, bo = x0 & 31;
    const uint32_t nmask = (1u << N) - 1u;

    R wb, wc, wa, wdv;
    ld_row(win + (int64_t)(j0 - 1) * P, wb);
    ld_row(win + (int64_t)j0 * P, wc);
    ld_row(win + (int64_t)(j0 + 1) * P, wa);
    ld_row_rw(wdp + (int64_t)j0 * P, wdv);
    T hl = win[(int64_t)j0 * P - 1];
    T hr = win[(int64_t)j0 * P + N];
    bool bad = false;

    for (int j = j0; j < j1; ++j) {
        // issue the next row's loads first
        R wn, wdn;
        T hln = (T)0, hrn = (T)0;
        const bool more = j + 1 < j1;
        if (more) {
            ld_row(win + (int64_t)(j + 2) * P, wn);
            ld_row_rw(wdp + (int64_t)(j + 1) * P, wdn);
            if (lane == 0) hln = win[(int64_t)(j + 1) * P - 1];
            if (lane == 31) hrn = win[(int64_t)(j + 1) * P + N];
        }
        T left0 = __shfl_up_sync(kFull, wc.v[N - 1], 1);
        T rightN = __shfl_down_sync(kFull, wc.v[0], 1);
        if (lane == 0) left0 = hl;
        if (lane == 31) rightN = hr;

        const uint8_t rf = a.rowflag[j];
        const bool special = (j == 0) | (j == ny - 1) | (rf != 0) | col_edge;
        R wnew, wdnew;
        if (!special) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                T wl = k == 0 ? left0 : wc.v[k - 1];
                T wr = k == N - 1 ? rightN : wc.v[k + 1];
                T lap = ((wa.v[k] + wb.v[k]) + (wl + wr)) - (T)4 * wc.v[k];
                wdnew.v[k] = wdv.v[k] + a.g * lap;
                wnew.v[k] = wc.v[k] + a.dt * wdnew.v[k];
            }
        } else {
            uint32_t vup = 0, vdn = 0, hcur = 0, hprev = 0;
            if (act) {
                if (rf & 2) vup = (a.cut_v[(int64_t)j * a.words + wi] >> bo) & nmask;
                if (rf & 4) {
                    const int jb = j > 0 ? j - 1 : ny - 1;
                    vdn = (a.cut_v[(int64_t)jb * a.words + wi] >> bo) & nmask;
                }
                if (rf & 1) {
                    hcur = (a.cut_h[(int64_t)j * a.words + wi] >> bo) & nmask;
                    if (x0 == 0) {
                        hprev = (a.cut_h[(int64_t)j * a.words + ((nx - 1) >> 5)] >> ((nx - 1) & 31)) & 1u;
                    } else if (bo == 0) {
                        hprev = a.cut_h[(int64_t)j * a.words + wi - 1] >> 31;
                    } else {
                        hprev = (a.cut_h[(int64_t)j * a.words + wi] >> (bo - 1)) & 1u;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int i = x0 + k;
                const T w0 = wc.v[k];
                T wl = k == 0 ? left0 : wc.v[k - 1];
                T wr = k == N - 1 ? rightN : wc.v[k + 1];
                T wu = wa.v[k], wdw = wb.v[k];
                // links to the row above / below
                if (j == ny - 1 && a.edge[TOP] != EDGE_PERIODIC) wu = edge_value(a.edge[TOP], ws[TOP], w0, wu);
                else if ((vup >> k) & 1u) wu = w0;
                if (j == 0 && a.edge[BOTTOM] != EDGE_PERIODIC) wdw = edge_value(a.edge[BOTTOM], ws[BOTTOM], w0, wdw);
                else if ((vdn >> k) & 1u) wdw = w0;
                // links to the west / east neighbour
                const uint32_t cut_w = k == 0 ? hprev : (hcur >> (k - 1)) & 1u;
                if (i == 0 && a.edge[LEFT] != EDGE_PERIODIC) wl = edge_value(a.edge[LEFT], ws[LEFT], w0, wl);
                else if (cut_w) wl = w0;
                if (i == nx - 1 && a.edge[RIGHT] != EDGE_PERIODIC) wr = edge_value(a.edge[RIGHT], ws[RIGHT], w0, wr);
                else if ((hcur >> k) & 1u) wr = w0;
                T lap = ((wu + wdw) + (wl + wr)) - (T)4 * w0;
                wdnew.v[k] = wdv.v[k] + a.g * lap;
                wnew.v[k] = w0 + a.dt * wdnew.v[k];
            }
        }

        if (act) {
            T *ro = wout + (int64_t)j * P;
            T *rd = wdp + (int64_t)j * P;
            if (x0 + N <= nx) {
                st_row(ro, wnew);
                st_row(rd, wdnew);
#pragma unroll
                for (int k = 0; k < N; ++k) bad |= !(isfinite(wnew.v[k]) && isfinite(wdnew.v[k]));
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k)
                    if (x0 + k < nx) {
                        ro[k] = wnew.v[k];
                        rd[k] = wdnew.v[k];
                        bad |= !(isfinite(wnew.v[k]) && isfinite(wdnew.v[k]));
                    }
            }
            // periodic images in the pads of the output buffer
            if (a.edge[TOP] == EDGE_PERIODIC) {
                if (j == 0) {
                    T *rp = wout + (int64_t)ny * P;
#pragma unroll
                    for (int k = 0; k < N; ++k) if (x0 + k < nx) rp[k] = wnew.v[k];
                }
                if (j == ny - 1) {
                    T *rp = wout - P;
#pragma unroll
                    for (int k = 0; k < N; ++k) if (x0 + k < nx) rp[k] = wnew.v[k];
                }
            }
            if (a.edge[LEFT] == EDGE_PERIODIC) {
                if (x0 == 0) ro[nx] = wnew.v[0];
#pragma unroll
                for (int k = 0; k < N; ++k) if (x0 + k == nx - 1) ro[-(x0 + 1)] = wnew.v[k];
            }
        }

        // rotate the register window
        wb = wc;
        wc = wa;
        if (more) {
            wa = wn;
            wdv = wdn;
            hl = hln;
            hr = hrn;
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(&a.st->err_bits, 1u);
}

template <typename T>
cudaError_t launch_bulk(const BulkArgs<T> &a, dim3 grid, cudaStream_t s)
{
    bulk_kernel<T><<<grid, kBulkThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ edge values

__device__ double load_value(const LoadDesc &L, int64_t n, double dt)
{
    const double t = (double)n * dt;
    switch (L.kind) {
    case LOAD_LINEAR:
        return (L.t <= 0.0 || t >= L.t) ? L.amp : L.amp * (t / L.t);
    case LOAD_SIN2: {
        if (L.t <= 0.0 || t >= L.t) return L.amp;
        const double sn = sin(kPi * t / (2.0 * L.t));
        return L.amp * sn * sn;
    }
    case LOAD_HALFSINE:
        return t >= L.t ? 0.0 : L.amp * sin(kPi * t / L.t);
    case LOAD_SERIES:
        if (L.n <= 0) return 0.0;
        return L.series[n < L.n ? n : L.n - 1];
    case LOAD_CONST:
        return L.amp;
    default:
        return 0.0;
    }
}

struct WstarArgs {
    CrackState *st;
    LoadDesc load[4];
    int32_t edge[4];
    double dt;
};

__global__ void wstar_kernel(const WstarArgs a)
{
    if (threadIdx.x < 4) {
        const int e = threadIdx.x;
        a.st->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], a.st->step, a.dt) : 0.0;
    }
}

cudaError_t launch_wstar(CrackState *st, const LoadDesc *load, const int32_t *edge, double dt, cudaStream_t s)
{
    WstarArgs a;
    a.st = st;
    for (int e = 0; e < 4; ++e) { a.load[e] = load[e]; a.edge[e] = edge[e]; }
    a.dt = dt;
    wstar_kernel<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------ periodic pad images

template <typename T>
__global__ void fill_pads_kernel(T *w, int64_t P, int nx, int ny, int xper, int yper)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (yper && t < nx) {
        w[(int64_t)ny * P + t] = w[t];                    // row ny <- row 0
        w[-P + t] = w[(int64_t)(ny - 1) * P + t];         // row -1 <- row ny-1
    }
    if (xper && t < ny) {
        w[(int64_t)t * P + nx] = w[(int64_t)t * P];       // column nx <- column 0
        w[(int64_t)t * P - 1] = w[(int64_t)t * P + nx - 1];
    }
}

template <typename T>
cudaError_t launch_fill_pads(T *w, int64_t pitch, int nx, int ny, const int32_t *edge, cudaStream_t s)
{
    const int xper = edge[LEFT] == EDGE_PERIODIC, yper = edge[BOTTOM] == EDGE_PERIODIC;
    if (!xper && !yper) return cudaSuccess;
    const int n = nx > ny ? nx : ny;
    fill_pads_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(w, pitch, nx, ny, xper, yper);
    return cudaGetLastError();
}

// ------------------------------------------------------------- crack step
//
// One CTA.  (1) Macroscopic crack-face rule (Sec. 3.1) on the boundary points
// of every severed crack link: for a lattice-aligned crack the normal through
// x_B is its column, x_I and x_II are the next two sites away from the face
// (distances 3/2 dh and 5/2 dh from it, x_B at 1/2 dh), and the quadratic
// p(s) = a + b s^2 with zero slope on the traction-free face gives
// w_B = (3 w_I - w_II) / 2; eq. f-macro-bc then makes wdot(x_B) =
// (w_B(t+dt) - w_B(t)) / dt.  (2) K_III by least squares of the crack opening
// over the site pairs straddling the crack at r in [r_min, r_min + W)
// (eq. sif, Sec. 4.2) in FP64 with a block reduction.  (3) Alg. 1: the
// criterion, the advance Delta a = adot dt on the 2^-32 dh grid, and the
// severing of the newly crossed links; then the history record and the
// Dirichlet values for the next step.
template <typename T>
__global__ void __launch_bounds__(kCrackThreads) crack_kernel(const CrackArgs<T> a)
{
    CrackState *st = a.st;
    const CrackParams &p = a.p;
    const int tid = threadIdx.x;
    const int64_t P = a.pitch;
    __shared__ double s_num[kCrackThreads / 32], s_den[kCrackThreads / 32];
    __shared__ int s_np[kCrackThreads / 32];

    const int i_first = st->i_first, i_last = st->i_last;
    if (p.mode != CRACK_NONE && p.macro && i_last >= i_first) {
        const int jc = p.jc;
        for (int c = i_first + tid; c <= i_last; c += kCrackThreads) {
            {   // below the crack: x_I = (c, jc-2), x_II = (c, jc-3)
                const T wI = a.w_out[(int64_t)(jc - 2) * P + c], wII = a.w_out[(int64_t)(jc - 3) * P + c];
                const T wB = (T)1.5 * wI - (T)0.5 * wII;
                const T wold = a.w_in[(int64_t)(jc - 1) * P + c];
                a.w_out[(int64_t)(jc - 1) * P + c] = wB;
                a.wd[(int64_t)(jc - 1) * P + c] = (wB - wold) / a.dt;
            }
            {   // above the crack: x_I = (c, jc+1), x_II = (c, jc+2)
                const T wI = a.w_out[(int64_t)(jc + 1) * P + c], wII = a.w_out[(int64_t)(jc + 2) * P + c];
                const T wB = (T)1.5 * wI - (T)0.5 * wII;
                const T wold = a.w_in[(int64_t)jc * P + c];
                a.w_out[(int64_t)jc * P + c] = wB;
                a.wd[(int64_t)jc * P + c] = (wB - wold) / a.dt;
            }
        }
    }
    __syncthreads();

    double r_min = 0.0, num = 0.0, den = 0.0;
    int np = 0;
    const int64_t tip = st->tip_q;
    if (p.mode != CRACK_NONE) {
        r_min = p.r_min_fixed > 0.0 ? p.r_min_fixed : p.r0 / (1.0 - st->v_prev);   // eq. r(v)
        const double lo = r_min / p.dh, hi = (r_min + p.fit_width) / p.dh;
        const double tip_h = (double)tip * kTwoM32;
        int c_lo = (int)floor(tip_h - hi - 0.5) - 1, c_hi = (int)floor(tip_h - lo - 0.5) + 1;
        c_lo = c_lo < i_first ? i_first : c_lo;
        c_hi = c_hi > i_last ? i_last : c_hi;
        const int jc = p.jc;
        for (int i = c_lo + tid; i <= c_hi; i += kCrackThreads) {
            if (!((a.cut_v[(int64_t)(jc - 1) * p.words + (i >> 5)] >> (i & 31)) & 1u)) continue;
            const double r_h = (double)(tip - ((int64_t)(2 * i + 1) << (kQBits - 1))) * kTwoM32;
            if (!(r_h >= lo && r_h < hi)) continue;
            const double r = r_h * p.dh;
            const double sf = sqrt(r / (2.0 * kPi));
            const double delta = (double)a.w_out[(int64_t)jc * P + i] - (double)a.w_out[(int64_t)(jc - 1) * P + i];
            num += delta * sf;
            den += sf * sf;
            ++np;
        }
    }
    // block reduction (warp shuffles, then one value per warp)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
        np += __shfl_down_sync(0xffffffffu, np, o);
    }
    if ((tid & 31) == 0) { s_num[tid >> 5] = num; s_den[tid >> 5] = den; s_np[tid >> 5] = np; }
    __syncthreads();
    if (tid != 0) return;
    num = 0.0; den = 0.0; np = 0;
    for (int q = 0; q < kCrackThreads / 32; ++q) { num += s_num[q]; den += s_den[q]; np += s_np[q]; }

    int32_t flags = st->flags;
    if (st->err_bits) flags |= FLAG_NONFINITE;
    if (p.mode != CRACK_NONE) {
        const double K = np > 0 ? p.mu / 4.0 * num / den : 0.0;
        int propagate = 0;
        double v = 0.0;
        if (p.mode == CRACK_PRESCRIBED) {
            propagate = 1;
            v = p.v_rel;
        } else if (p.mode == CRACK_KCRIT && np > 0 && fabs(K) > p.K_C) {
            const double ratio = fabs(K) / p.K_C;
            propagate = 1;
            v = p.v_max * tanh(sqrt(ratio * ratio * ratio * ratio - 1.0));   // eq. v-tanh
        }
        if (!isfinite(K)) flags |= FLAG_NONFINITE;
        if (st->arrested) { propagate = 0; v = 0.0; }
        int grew = 0;
        int64_t tip_new = tip;
        if (propagate) {
            const double adot = v * p.cs;
            const int64_t dq = __double2ll_rn(adot * p.dt / p.dh * 4294967296.0);   // Delta a = adot dt
            int64_t next = tip + dq;
            if (next >= p.clamp_q) { next = p.clamp_q; st->arrested = 1; flags |= FLAG_CLAMPED; }
            if (next > tip) {
                // links at x_i = (i + 1/2) dh with tip < x_i <= next are crossed by the new segment
                int64_t last = (next - ((int64_t)1 << (kQBits - 1))) >> kQBits;
                if (last > p.nx - 1) last = p.nx - 1;
                const int jr = p.jc - 1;
                for (int64_t i = (int64_t)i_last + 1; i <= last; ++i) {
                    if (i < i_first) continue;
                    a.cut_v[(int64_t)jr * p.words + (i >> 5)] |= 1u << (i & 31);
                }
                if (last > i_last && last >= i_first) {
                    st->i_last = (int32_t)last;
                    a.rowflag[jr] |= 2;
                    a.rowflag[jr + 1] |= 4;
                }
                tip_new = next;
                grew = 1;
            }
        }
        st->tip_q = tip_new;
        st->v_prev = p.mode == CRACK_PRESCRIBED ? p.v_rel : v;
        st->K = K;
        st->v = v;
        st->r_min = r_min;
        st->npairs = np;
        st->grew = grew;
        if (p.hist_cap > 0) {
            const int64_t h = st->hist_n % p.hist_cap;
            a.hist.K[h] = K;
            a.hist.v[h] = v;
            a.hist.tip[h] = tip_new;
            a.hist.np[h] = np;
        }
        st->hist_n += 1;
    }
    st->flags = flags;
    const int64_t n = st->step + 1;
    st->step = n;
    for (int e = 0; e < 4; ++e)
        st->wstar[e] = a.edge[e] == EDGE_DIRICHLET ? load_value(a.load[e], n, (double)p.dt) : 0.0;
}

template <typename T>
cudaError_t launch_crack(const CrackArgs<T> &a, cudaStream_t s)
{
    crack_kernel<T><<<1, kCrackThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_bulk<float>(const BulkArgs<float> &, dim3, cudaStream_t);
template cudaError_t launch_bulk<double>(const BulkArgs<double> &, dim3, cudaStream_t);
template cudaError_t launch_crack<float>(const CrackArgs<float> &, cudaStream_t);
template cudaError_t launch_crack<double>(const CrackArgs<double> &, cudaStream_t);
template cudaError_t launch_fill_pads<float>(float *, int64_t, int, int, const int32_t *, cudaStream_t);
template cudaError_t launch_fill_pads<double>(double *, int64_t, int, int, const int32_t *, cudaStream_t);

}  // namespace lbm
