// lbm_rows.cuh -- per-thread row helpers shared by the time-step kernel and
// its adjoint: 16-byte vector loads and stores of a row segment, the storage
// forms of wdot, the pad images of the edge sites, and the update of one row
// segment with every boundary rule (the moment form of Sec. 3 with the
// link-local rules of Sec. 3.1).
#pragma once

#include "lbm_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <type_traits>

namespace lbm {

// --------------------------------------------------------- vector rows

template <typename T, int N> struct Row { T v[N]; };

// w of the input buffer is read-only during a step: non-coherent loads.
__device__ __forceinline__ void ldg_row(const float *p, Row<float, 4> &r)
{
    float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
}
__device__ __forceinline__ void ldg_row(const double *p, Row<double, 2> &r)
{
    double2 q = __ldg(reinterpret_cast<const double2 *>(p));
    r.v[0] = q.x; r.v[1] = q.y;
}
// wdot is updated in place: coherent loads.
__device__ __forceinline__ void ld_row(const float *p, Row<float, 4> &r)
{
    float4 q = *reinterpret_cast<const float4 *>(p);
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
}
__device__ __forceinline__ void ld_row(const double *p, Row<double, 2> &r)
{
    double2 q = *reinterpret_cast<const double2 *>(p);
    r.v[0] = q.x; r.v[1] = q.y;
}
// w of the input buffer: through the read-only path (NC), or with coherent
// loads when the same launch wrote it (a persistent kernel that steps many
// times, whose grid barrier orders the steps' stores and loads).
template <bool COH, typename T, int N>
__device__ __forceinline__ void load_w(const T *p, Row<T, N> &r)
{
    if (COH) ld_row(p, r);
    else ldg_row(p, r);
}
__device__ __forceinline__ void stg_row(float *p, const Row<float, 4> &r)
{
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
}
__device__ __forceinline__ void stg_row(double *p, const Row<double, 2> &r)
{
    *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
}

// Storage of wdot.  FP64 and FP32 store the value; the 16-bit forms store
// wdot * scale rounded to nearest (BF16: scale 1; FP16: a power of two chosen
// so that the values sit well inside FP16's range), arithmetic stays FP32.
// fetch() issues the load of a row into its raw form and unpack() converts
// it, so that a march can keep a 16-bit row in flight for a whole iteration
// (converting right after the load would wait for it there).
template <typename D> struct WdIO;
template <> struct WdIO<double> {
    typedef Row<double, 2> Raw;
    static __device__ __forceinline__ void fetch(const double *p, Raw &r) { ld_row(p, r); }
    static __device__ __forceinline__ void unpack(const Raw &q, Row<double, 2> &r, double) { r = q; }
    static __device__ __forceinline__ void load(const double *p, Row<double, 2> &r, double) { ld_row(p, r); }
    static __device__ __forceinline__ void store(double *p, const Row<double, 2> &r, double) { stg_row(p, r); }
    static __device__ __forceinline__ void put(double *p, double v, double) { *p = v; }
};
template <> struct WdIO<float> {
    typedef Row<float, 4> Raw;
    static __device__ __forceinline__ void fetch(const float *p, Raw &r) { ld_row(p, r); }
    static __device__ __forceinline__ void unpack(const Raw &q, Row<float, 4> &r, float) { r = q; }
    static __device__ __forceinline__ void load(const float *p, Row<float, 4> &r, float) { ld_row(p, r); }
    static __device__ __forceinline__ void store(float *p, const Row<float, 4> &r, float) { stg_row(p, r); }
    static __device__ __forceinline__ void put(float *p, float v, float) { *p = v; }
};
template <> struct WdIO<__nv_bfloat16> {
    typedef uint2 Raw;
    static __device__ __forceinline__ void fetch(const __nv_bfloat16 *p, Raw &q) { q = *reinterpret_cast<const uint2 *>(p); }
    static __device__ __forceinline__ void unpack(const Raw &q, Row<float, 4> &r, float)
    {
        r.v[0] = __uint_as_float(q.x << 16);
        r.v[1] = __uint_as_float(q.x & 0xffff0000u);
        r.v[2] = __uint_as_float(q.y << 16);
        r.v[3] = __uint_as_float(q.y & 0xffff0000u);
    }
    static __device__ __forceinline__ void load(const __nv_bfloat16 *p, Row<float, 4> &r, float s)
    {
        Raw q;
        fetch(p, q);
        unpack(q, r, s);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, const Row<float, 4> &r, float)
    {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(r.v[0], r.v[1]);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(r.v[2], r.v[3]);
        uint2 q;
        q.x = *reinterpret_cast<const uint32_t *>(&lo);
        q.y = *reinterpret_cast<const uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(p) = q;
    }
    static __device__ __forceinline__ void put(__nv_bfloat16 *p, float v, float) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float get(const __nv_bfloat16 *p, float) { return __bfloat162float(*p); }
};
template <> struct WdIO<__half> {
    // scale: stored = wdot * scale; loads multiply by 1 / scale (both exact powers of two)
    typedef uint2 Raw;
    static __device__ __forceinline__ void fetch(const __half *p, Raw &q) { q = *reinterpret_cast<const uint2 *>(p); }
    static __device__ __forceinline__ void load(const __half *p, Row<float, 4> &r, float inv)
    {
        Raw q;
        fetch(p, q);
        unpack(q, r, inv);
    }
    static __device__ __forceinline__ void unpack(const Raw &q, Row<float, 4> &r, float inv)
    {
        const __half2 lo = *reinterpret_cast<const __half2 *>(&q.x);
        const __half2 hi = *reinterpret_cast<const __half2 *>(&q.y);
        const float2 a = __half22float2(lo), b = __half22float2(hi);
        r.v[0] = a.x * inv;
        r.v[1] = a.y * inv;
        r.v[2] = b.x * inv;
        r.v[3] = b.y * inv;
    }
    static __device__ __forceinline__ void store(__half *p, const Row<float, 4> &r, float scale)
    {
        const __half2 lo = __floats2half2_rn(r.v[0] * scale, r.v[1] * scale);
        const __half2 hi = __floats2half2_rn(r.v[2] * scale, r.v[3] * scale);
        uint2 q;
        q.x = *reinterpret_cast<const uint32_t *>(&lo);
        q.y = *reinterpret_cast<const uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(p) = q;
    }
    static __device__ __forceinline__ void put(__half *p, float v, float scale) { *p = __float2half_rn(v * scale); }
    static __device__ __forceinline__ float get(const __half *p, float inv) { return __half2float(*p) * inv; }
};


// Leapfrog storage (LBM_F32_LEAPFROG).  With the Euler integration of Sec. 3
// (eq. integration) wdot_n = (w_n - w_{n-1}) / dt exactly, so the state can
// be kept as the two FP32 planes w_n and w_{n-1} instead of w and wdot: the
// step reads w_n (with its neighbours) and w_{n-1} and overwrites w_{n-1}
// with w_{n+1} = w_n + ((w_n - w_{n-1}) + g dt lap), 12 bytes per site
// instead of 16.  Its "wdot plane" is the previous w, i.e. the output
// buffer of the step: loads of it read w_{n-1}, and wdot is never stored.
template <> struct WdIO<Lf> {
    typedef Row<float, 4> Raw;
    static __device__ __forceinline__ void fetch(const Lf *p, Raw &r) { ld_row(reinterpret_cast<const float *>(p), r); }
    static __device__ __forceinline__ void unpack(const Raw &q, Row<float, 4> &r, float) { r = q; }
    static __device__ __forceinline__ void load(const Lf *p, Row<float, 4> &r, float)
    {
        ld_row(reinterpret_cast<const float *>(p), r);
    }
    static __device__ __forceinline__ void store(Lf *, const Row<float, 4> &, float) {}
    static __device__ __forceinline__ void put(Lf *, float, float) {}
};

// One site's update: wdot' = wdot + g lap, w' = w + dt wdot' (moment form),
// or, with leapfrog storage (the second argument is then w_{n-1}),
// w' = w + ((w - w_{n-1}) + g dt lap).
template <typename T, typename D>
__device__ __forceinline__ void site_update(T w0, T wdv, T lap, T g, T dt, T &wnew, T &wdnew)
{
    if constexpr (std::is_same<D, Lf>::value) {
        wnew = w0 + ((w0 - wdv) + (g * dt) * lap);
        wdnew = wnew;
    } else {
        wdnew = wdv + g * lap;
        wnew = w0 + dt * wdnew;
    }
}

// Pad images of the new values of row j, for the next step's neighbours.
template <typename A, typename T, int N>
__device__ __forceinline__ void write_pads(const A &a, int x0, int j, const Row<T, N> &wnew)
{
    const int nx = a.nx, ny = a.ny;
    const int64_t P = a.pitch;
    const int eL = a.edge[LEFT], eR = a.edge[RIGHT], eB = a.edge[BOTTOM], eT = a.edge[TOP];
    T *row = a.w_out + (int64_t)j * P;   // column 0 of row j
    if (x0 == 0) {
        if (eL == EDGE_FREE) row[-1] = wnew.v[0];
        else if (eL == EDGE_PERIODIC) row[nx] = wnew.v[0];
    }
    const int kr = nx - 1 - x0;
    if (kr >= 0 && kr < N) {
        T v = wnew.v[0];
#pragma unroll
        for (int k = 1; k < N; ++k) if (k == kr) v = wnew.v[k];
        if (eR == EDGE_FREE) row[nx] = v;
        else if (eR == EDGE_PERIODIC) row[-1] = v;
    }
    if (j == 0 || j == ny - 1) {
        T *pr = nullptr;
        if (j == 0 && eB == EDGE_FREE) pr = row - P;
        else if (j == 0 && eB == EDGE_PERIODIC) pr = a.w_out + (int64_t)ny * P;
        if (j == ny - 1 && eT == EDGE_FREE) pr = row + P;
        else if (j == ny - 1 && eT == EDGE_PERIODIC) pr = a.w_out - P;
        if (pr) {
#pragma unroll
            for (int k = 0; k < N; ++k) if (x0 + k < nx) pr[x0 + k] = wnew.v[k];
        }
    }
}

// Store row j of the new fields (masked at the right end of the lattice).
template <typename A, typename T, int N>
__device__ __forceinline__ void store_row(const A &a, int x0, int j, const Row<T, N> &wnew,
                                          const Row<T, N> &wdnew, T &acc)
{
    typedef typename std::remove_pointer<decltype(a.wd)>::type D;
    const int64_t o = (int64_t)j * a.pitch + x0;
    if (x0 + N <= a.nx) {
        stg_row(a.w_out + o, wnew);
        WdIO<D>::store(a.wd + o, wdnew, a.wd_scale);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (x0 + k < a.nx) {
                a.w_out[o + k] = wnew.v[k];
                WdIO<D>::put(a.wd + o + k, wdnew.v[k], a.wd_scale);
            }
    }
    acc += wnew.v[0];
}

// Twice the Dirichlet value of each edge at t_n (anti-bounce-back sends 2 w* - w),
// read once per CTA.
template <typename T> struct EdgeValues { T two_ws[4]; };

template <typename T>
__device__ __forceinline__ EdgeValues<T> edge_values(const CrackState *s_in)
{
    EdgeValues<T> E;
#pragma unroll
    for (int e = 0; e < 4; ++e) E.two_ws[e] = (T)2 * (T)s_in->wstar[e];
    return E;
}

// One row of the update with every boundary rule: Dirichlet edges
// (anti-bounce-back, value 2 w* - w), severed links to the row above (cut_up)
// and below (cut_dn) (bounce-back, value w); free and periodic edges come in
// through the pads.
template <typename A, typename T, int N>
__device__ __forceinline__ void row_update(const A &a, const EdgeValues<T> &E, int x0, int j, const Row<T, N> &wc,
                                           const Row<T, N> &up0, const Row<T, N> &dn0, const Row<T, N> &wdv, T left0,
                                           T rightN, uint32_t cut_up, uint32_t cut_dn, Row<T, N> &wnew,
                                           Row<T, N> &wdnew)
{
    const int nx = a.nx, ny = a.ny;
    const bool dir_t = j == ny - 1 && a.edge[TOP] == EDGE_DIRICHLET;
    const bool dir_b = j == 0 && a.edge[BOTTOM] == EDGE_DIRICHLET;
    const bool dir_l = a.edge[LEFT] == EDGE_DIRICHLET, dir_r = a.edge[RIGHT] == EDGE_DIRICHLET;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const T w0 = wc.v[k];
        T wl = k == 0 ? left0 : wc.v[k - 1];
        T wr = k == N - 1 ? rightN : wc.v[k + 1];
        T up = up0.v[k], dn = dn0.v[k];
        if (dir_t) up = E.two_ws[TOP] - w0;
        else if ((cut_up >> k) & 1u) up = w0;
        if (dir_b) dn = E.two_ws[BOTTOM] - w0;
        else if ((cut_dn >> k) & 1u) dn = w0;
        if (dir_l && x0 + k == 0) wl = E.two_ws[LEFT] - w0;
        if (dir_r && x0 + k == nx - 1) wr = E.two_ws[RIGHT] - w0;
        const T lap = ((up + dn) + (wl + wr)) - (T)4 * w0;
        typedef typename std::remove_pointer<decltype(a.wd)>::type D;
        site_update<T, D>(w0, wdv.v[k], lap, a.g, a.dt, wnew.v[k], wdnew.v[k]);
    }
}

}  // namespace lbm
