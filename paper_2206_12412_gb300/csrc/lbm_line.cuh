// lbm_line.cuh -- the tabulated boundary points of the macroscopic rule on
// the faces of a crack in any direction, shared by the host runtime that
// builds the table and the kernel that applies it.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// One site that the macroscopic rule (Sec. 3.1) may govern: a site within
// 1.5 spacings of the crack's line.  It takes the line's normal n, pointing
// away from the line; x_I = x_B + n dh and x_II = x_B + 2 n dh are
// interpolated bilinearly (their cells' corners all lie on x_B's side), and
// the quadratic with zero slope at the line gives
// w_B = sum_k a_k w(corner_k): the I corners weighted by
// (s_II^2 - s_B^2) / (s_II^2 - s_I^2), the II corners by
// (s_B^2 - s_I^2) / (s_II^2 - s_I^2), s the distances from the line.
// Unused corners have a_k = 0; cand[k] is the corner's index in the table
// (-1: not a tabulated site).  The rule applies to the site once one of its
// links is severed.
struct LineFace {
    int32_t i, j;
    int32_t ci[8], cj[8], cand[8];
    double a[8];
};

// The device scratch of the face solve, per tabulated point: two sweeps'
// values (used when the points outnumber the kernel's shared memory), the
// fixed part of each point's sum, the list of points, each table entry's
// position in it (-1: not a point), the mask of coupled corners and their
// list positions.
struct FaceScratch {
    double *buf_a, *buf_b, *base;
    int32_t *list, *pos;
    uint32_t *mask;
    int32_t *kpos;
};
constexpr size_t kLineFaceScratch = 3 * sizeof(double) + 3 * sizeof(int32_t) + 8 * sizeof(int32_t);

template <typename T, typename D>
cudaError_t launch_line_faces(const StepArgs<T, D> &a, const LineFace *faces, int nf, double *scratch, cudaStream_t s);

}  // namespace lbm
