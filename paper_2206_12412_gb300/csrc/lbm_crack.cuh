// lbm_crack.cuh -- device code shared by the time-step kernels: the
// boundary value of a Dirichlet edge and the warp-collective crack step of
// Alg. 1 for one end of the crack.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// ------------------------------------------------------------ edge values

__device__ __forceinline__ double load_value(const LoadDesc L, int64_t n, double dt)
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

// ------------------------------------------------------------ crack step
//
// Warp-collective crack handling of Alg. 1 for one end of the crack (dir =
// +1: the right end, growing towards +x; -1: the left end of a two-tip
// crack, growing towards -x) of the state S (in shared memory), given the
// fields w after the LBM step.  (1) K_III by least squares of the crack
// opening over the site pairs straddling the crack at r in [r_min, r_min + W)
// behind the tip (eq. sif; Sec. 4.2 and eq. r(v) with this end's previous
// speed), in FP64 with a warp reduction.  (2) The criterion: prescribed
// growth, or |K| > K_C with v = v_max tanh(sqrt((K/K_C)^4 - 1)) (eq.
// v-tanh).  (3) The advance Delta a = adot dt, rounded to the 2^-32 dh grid;
// the links at x_i = (i + 1/2) dh between the old and the new tip are
// severed (closed segment); the right end stops at x = nx dh, the left at 0.
// Lane 0 updates this end's fields of S (and i_last or i_first) and the cut
// mask and, if `commit`, writes this end's history record at hist_n (the
// caller advances hist_n once per crack step).  Two CTAs may run it on the
// same state at once: both reach the same decision and set the same bits.

// The least-squares sums of step (1) for one end: num = sum delta_i s_i,
// den = sum s_i^2 over the np pairs in the window, and the window's r_min.
struct CrackSums {
    double num, den, r_min;
    int np;
};

// Step (1) for one end, by a group of G lanes (32: a warp; 16: a half warp,
// so that one warp evaluates both ends at once); every lane of the group
// gets the sums.  Reads S only.  All 32 lanes of the warp must call it.
template <typename T, int G = 32>
__device__ __forceinline__ CrackSums crack_eval_warp(const CrackParams &p, const T *w, int64_t P, const uint32_t *cut_v,
                                                     const CrackState &S, int dir)
{
    const int lane = threadIdx.x & (G - 1);
    const TipState &E = dir > 0 ? S.r : S.l;
    const int64_t tip = E.tip_q;
    const int i_first = S.i_first, i_last = S.i_last;
    // eq. r(v); the divisions are skipped where they are exact (v = 0, dh = 1):
    // FP64 instructions are few per cycle on GB300, and this chain is on
    // the crack step's critical path
    const double r_min = p.r_min_fixed > 0.0 ? p.r_min_fixed : (E.v_prev == 0.0 ? p.r0 : p.r0 / (1.0 - E.v_prev));
    const double lo = p.dh == 1.0 ? r_min : r_min / p.dh;
    const double hi = p.dh == 1.0 ? r_min + p.fit_width : (r_min + p.fit_width) / p.dh;
    const double tip_h = (double)tip * kTwoM32;
    int c_lo, c_hi;
    if (dir > 0) {
        c_lo = (int)floor(tip_h - hi - 0.5) - 1;
        c_hi = (int)floor(tip_h - lo - 0.5) + 1;
    } else {
        c_lo = (int)floor(tip_h + lo - 0.5) - 1;
        c_hi = (int)floor(tip_h + hi - 0.5) + 1;
    }
    c_lo = c_lo < i_first ? i_first : c_lo;
    c_hi = c_hi > i_last ? i_last : c_hi;
    const int jc = p.jc;
    double num = 0.0, den = 0.0;
    int np = 0;
    for (int i = c_lo + lane; i <= c_hi; i += G) {
        // the pair's fields are loaded together with its mask word (the
        // columns lie in [i_first, i_last], inside the lattice), so the two
        // loads cost one round trip
        const uint32_t word = cut_v[(int64_t)(jc - 1) * p.words + (i >> 5)];
        const T above = w[(int64_t)jc * P + i], below = w[(int64_t)(jc - 1) * P + i];
        if (!((word >> (i & 31)) & 1u)) continue;
        const int64_t xq = (int64_t)(2 * i + 1) << (kQBits - 1);
        const double r_h = (double)(dir > 0 ? tip - xq : xq - tip) * kTwoM32;
        if (!(r_h >= lo && r_h < hi)) continue;
        const double r = p.dh == 1.0 ? r_h : r_h * p.dh;
        const double sf = sqrt(r / (2.0 * kPi));
        const double delta = (double)above - (double)below;
        num += delta * sf;
        den += sf * sf;
        ++np;
    }
    // with the pairs in one lane of the group (the one-pair window W = dh
    // always), that lane's sums are the group's: adding the other lanes'
    // zeros cannot change them, so one shuffle replaces the reduction tree
    const unsigned gmask = G == 32 ? 0xffffffffu : (0xffffu << (threadIdx.x & 16));
    const unsigned holders = __ballot_sync(0xffffffffu, np > 0) & gmask;
    if (__popc(holders) <= 1) {
        const int src = holders ? __ffs(holders) - 1 : (threadIdx.x & 31 & ~(G - 1));
        num = __shfl_sync(0xffffffffu, num, src);
        den = __shfl_sync(0xffffffffu, den, src);
        np = __shfl_sync(0xffffffffu, np, src);
        return CrackSums{num, den, r_min, np};
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
        np += __shfl_xor_sync(0xffffffffu, np, o);
    }
    return CrackSums{num, den, r_min, np};
}

// K from the sums (eq. sif; least squares when the window holds several
// pairs) and step (2), the criterion, for one end: the FP64 part of the
// crack step, which reads this end's state only (so the two ends of a
// two-tip crack can decide at once, in different lanes).
struct CrackDecision {
    double K, v;
    int64_t dq;          // the advance on the 2^-32 dh grid (propagate only)
    int32_t propagate, flags;
};

__device__ __forceinline__ CrackDecision crack_decide(const CrackParams &p, const CrackState &S, int dir,
                                                      const CrackSums &c)
{
    const double K = c.np > 0 ? p.mu / 4.0 * c.num / c.den : 0.0;
    const TipState &E = dir > 0 ? S.r : S.l;
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
    if (E.arrested) { propagate = 0; v = 0.0; }
    // Delta a = adot dt on the 2^-32 dh grid (prescribed growth: the step the
    // host formed with the same expression, once)
    int64_t dq = p.dq_prescribed;
    if (propagate && p.mode != CRACK_PRESCRIBED) {
        const double adot = v * p.cs;
        const double a1 = p.dt == 1.0 ? adot : adot * p.dt;
        dq = __double2ll_rn((p.dh == 1.0 ? a1 : a1 / p.dh) * 4294967296.0);
    }
    return CrackDecision{K, v, dq, propagate, flags};
}

// Step (3) for one end, by one thread: the advance, the severed links, this
// end's fields of S and, if `commit`, its history record.
__device__ __forceinline__ void crack_commit(const CrackParams &p, uint32_t *cut_v, const History &hist, CrackState &S,
                                             int dir, bool commit, const CrackSums &c, const CrackDecision &d)
{
    const double K = d.K, v = d.v;
    const int np = c.np;
    const double r_min = c.r_min;
    TipState &E = dir > 0 ? S.r : S.l;
    const int64_t tip = E.tip_q;
    const int i_first = S.i_first, i_last = S.i_last;
    const int propagate = d.propagate;
    int32_t flags = d.flags;
    int grew = 0;
    int64_t tip_new = tip;
    const int jr = p.jc - 1;
    const int64_t half = (int64_t)1 << (kQBits - 1);
    if (propagate) {
        const int64_t dq = d.dq;
        if (dir > 0) {
            int64_t next = tip + dq;
            if (next >= p.clamp_q) { next = p.clamp_q; E.arrested = 1; flags |= FLAG_CLAMPED; }
            if (next > tip) {
                int64_t last = (next - half) >> kQBits;   // largest i with x_i <= next
                if (last > p.nx - 1) last = p.nx - 1;
                for (int64_t i = (int64_t)i_last + 1; i <= last; ++i) {
                    if (i < i_first) continue;
                    atomicOr(&cut_v[(int64_t)jr * p.words + (i >> 5)], 1u << (i & 31));
                }
                if (last > i_last && last >= i_first) S.i_last = (int32_t)last;
                tip_new = next;
                grew = 1;
            }
        } else {
            int64_t next = tip - dq;
            if (next <= 0) { next = 0; E.arrested = 1; flags |= FLAG_CLAMPED; }
            if (next < tip) {
                int64_t first = (next - half + ((int64_t)1 << kQBits) - 1) >> kQBits;   // smallest i with x_i >= next
                if (first < 0) first = 0;
                for (int64_t i = first; i < (int64_t)i_first; ++i) {
                    if (i > i_last) continue;
                    atomicOr(&cut_v[(int64_t)jr * p.words + (i >> 5)], 1u << (i & 31));
                }
                if (first < i_first && first <= i_last) S.i_first = (int32_t)first;
                tip_new = next;
                grew = 1;
            }
        }
    }
    E.tip_q = tip_new;
    E.v_prev = p.mode == CRACK_PRESCRIBED ? p.v_rel : v;
    E.K = K;
    E.v = v;
    E.r_min = r_min;
    E.npairs = np;
    E.grew = grew;
    E.flags = flags;
    if (commit && p.hist_cap > 0) {
        const int64_t h = S.hist_n % p.hist_cap;
        if (dir > 0) {
            hist.K[h] = K;
            hist.v[h] = v;
            hist.tip[h] = tip_new;
            hist.np[h] = np;
        } else {
            hist.Kl[h] = K;
            hist.vl[h] = v;
            hist.tipl[h] = tip_new;
            hist.npl[h] = np;
        }
    }
    E.decided = 1;
}


__device__ __forceinline__ void crack_apply(const CrackParams &p, uint32_t *cut_v, const History &hist, CrackState &S,
                                            int dir, bool commit, const CrackSums &c)
{
    crack_commit(p, cut_v, hist, S, dir, commit, c, crack_decide(p, S, dir, c));
}

// Prescribed growth whose K fit the step kernel's record CTA forms
// (crack_record_prescribed): the decision of Alg. 1 needs no K -- the speed
// is given, so eq. r(v) and the advance use it -- and this end advances at
// once, by one thread: the severed links, this end's fields of S but K, r_min
// and the pair count, and, if `commit`, its history's tip and speed.
__device__ __forceinline__ void crack_advance_prescribed(const CrackParams &p, uint32_t *cut_v, const History &hist,
                                                         CrackState &S, int dir, bool commit)
{
    TipState &E = dir > 0 ? S.r : S.l;
    if (p.mode == CRACK_NONE || E.decided) {
        E.decided = 1;
        return;
    }
    CrackDecision d;
    d.K = 0.0;
    d.v = E.arrested ? 0.0 : p.v_rel;
    d.dq = p.dq_prescribed;
    d.propagate = E.arrested ? 0 : 1;
    d.flags = E.flags;
    const CrackSums c = {0.0, 0.0, 0.0, 0};
    const int64_t h = p.hist_cap > 0 ? S.hist_n % p.hist_cap : 0;
    crack_commit(p, cut_v, hist, S, dir, false, c, d);
    if (commit && p.hist_cap > 0) {
        if (dir > 0) {
            hist.v[h] = d.v;
            hist.tip[h] = E.tip_q;
        } else {
            hist.vl[h] = d.v;
            hist.tipl[h] = E.tip_q;
        }
    }
}

// The fields of this end's decision that crack_advance_prescribed forms (all
// of the state's end but K, r_min and the pair count).
__device__ __forceinline__ void copy_tip_decision(TipState &o, const TipState &s)
{
    o.tip_q = s.tip_q;
    o.tip_yq = s.tip_yq;
    o.arrested = s.arrested;
    o.grew = s.grew;
    o.flags = s.flags;
    o.v_prev = s.v_prev;
    o.v = s.v;
}

// The other half of a prescribed-growth crack step, by one warp of a CTA
// that updates no rows: the K fit of eq. sif from the state before the step
// (S_old, as crack_step_warp reads it) and the fields the step follows -- the
// same sums in the same order, so the same K -- written to this end's K,
// r_min and pair count in S_out and to the history.  A non-finite K sets the
// launch's error word.  All 32 lanes must call it.
template <typename T>
__device__ __forceinline__ void crack_record_prescribed(const CrackParams &p, const T *w, int64_t P,
                                                        const uint32_t *cut_v, const History &hist,
                                                        const CrackState &S_old, CrackState *S_out, uint32_t *err,
                                                        int dir)
{
    const TipState &E = dir > 0 ? S_old.r : S_old.l;
    TipState &O = dir > 0 ? S_out->r : S_out->l;
    if (E.decided) {
        // applied already (a deferred crack step before a host read): carry
        // its K over, as the advancing CTA carries the rest of the state
        if ((threadIdx.x & 31) == 0) {
            O.K = E.K;
            O.r_min = E.r_min;
            O.npairs = E.npairs;
        }
        return;
    }
    // the window lies behind the old tip, where every link is severed
    // already: the bits the advancing CTA sets meanwhile are not read
    const CrackSums c = crack_eval_warp<T>(p, w, P, cut_v, S_old, dir);
    if ((threadIdx.x & 31) == 0) {
        const double K = c.np > 0 ? p.mu / 4.0 * c.num / c.den : 0.0;
        O.K = K;
        O.r_min = c.r_min;
        O.npairs = c.np;
        if (!isfinite(K)) atomicOr(err, (uint32_t)ERR_NONFINITE);
        if (p.hist_cap > 0) {
            const int64_t h = S_old.hist_n % p.hist_cap;
            if (dir > 0) {
                hist.K[h] = K;
                hist.np[h] = c.np;
            } else {
                hist.Kl[h] = K;
                hist.npl[h] = c.np;
            }
        }
    }
}

// Whether the pending crack step of S can sever a link: an end that still
// grows (not decided, not arrested) reaches the centre of the next link it
// would sever if it advanced by p.dq_max, more than any step of the
// K-criterion advances.  When it cannot, the rows next to the crack do not
// depend on the step's decision (only its state and history do).
__device__ __forceinline__ bool crack_cut_in_reach(const CrackParams &p, const CrackState &S)
{
    const int64_t half = (int64_t)1 << (kQBits - 1);
    bool reach = false;
    if (!S.r.decided && !S.r.arrested) {
        // the first column a right-end advance can sever
        const int64_t i = max((int64_t)S.i_last + 1, (int64_t)S.i_first);
        if (i <= p.nx - 1) reach |= ((2 * i + 1) * half) <= S.r.tip_q + p.dq_max;
    }
    if (p.two_tips && !S.l.decided && !S.l.arrested) {
        // the first column a left-end advance can sever
        const int64_t i = min((int64_t)S.i_first - 1, (int64_t)S.i_last);
        if (i >= 0) reach |= ((2 * i + 1) * half) >= S.l.tip_q - p.dq_max;
    }
    return reach;
}

// The crack step of both ends of a two-tip crack by one warp: lanes 0-15
// evaluate the right end and lanes 16-31 the left end at once, on the same
// state (the criteria of both ends before either advances); lane 0 then
// advances the right end and the left end in turn.
template <typename T>
__device__ __forceinline__ void crack_step_both(const CrackParams &p, const T *w, int64_t P, uint32_t *cut_v,
                                                const History &hist, CrackState &S, bool commit)
{
    const int lane = threadIdx.x & 31;
    const bool act_r = p.mode != CRACK_NONE && !S.r.decided;
    const bool act_l = p.mode != CRACK_NONE && !S.l.decided;
    const CrackSums c = crack_eval_warp<T, 16>(p, w, P, cut_v, S, lane < 16 ? +1 : -1);
    // each end's criterion (the FP64 part) in its half warp's first lane at
    // once: lane 0 the right end, lane 16 the left end
    CrackDecision dd = {};
    if ((lane & 15) == 0) dd = crack_decide(p, S, lane < 16 ? +1 : -1, c);
    CrackSums cl;
    cl.num = __shfl_sync(0xffffffffu, c.num, 16);
    cl.den = __shfl_sync(0xffffffffu, c.den, 16);
    cl.r_min = __shfl_sync(0xffffffffu, c.r_min, 16);
    cl.np = __shfl_sync(0xffffffffu, c.np, 16);
    CrackDecision dl;
    dl.K = __shfl_sync(0xffffffffu, dd.K, 16);
    dl.v = __shfl_sync(0xffffffffu, dd.v, 16);
    dl.dq = __shfl_sync(0xffffffffu, dd.dq, 16);
    dl.propagate = __shfl_sync(0xffffffffu, dd.propagate, 16);
    dl.flags = __shfl_sync(0xffffffffu, dd.flags, 16);
    if (lane == 0) {
        if (act_r) crack_commit(p, cut_v, hist, S, +1, commit, c, dd);
        if (act_l) crack_commit(p, cut_v, hist, S, -1, commit, cl, dl);
        S.r.decided = 1;
        S.l.decided = 1;
    }
    __syncwarp();
}

// Both steps for one end, by one warp (lane 0 applies).
template <typename T>
__device__ __forceinline__ void crack_step_warp(const CrackParams &p, const T *w, int64_t P, uint32_t *cut_v,
                                                const History &hist, CrackState &S, int dir, bool commit)
{
    const int lane = threadIdx.x & 31;
    TipState &E = dir > 0 ? S.r : S.l;
    if (p.mode == CRACK_NONE || E.decided) {
        __syncwarp();
        if (lane == 0) E.decided = 1;
        __syncwarp();
        return;
    }
    const CrackSums c = crack_eval_warp<T>(p, w, P, cut_v, S, dir);
    if (lane == 0) crack_apply(p, cut_v, hist, S, dir, commit, c);
    __syncwarp();
}

}  // namespace lbm
