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
// flags bit FACE_DROPPED: a stencil of the point has a corner outside the
// body and was left out (the rule is not supported there; the solve reports
// FLAG_UNSUPPORTED once such a point is governed by the rule).
struct LineFace {
    int32_t i, j;
    int32_t ci[8], cj[8], cand[8];
    int32_t flags, pad;
    double a[8];
    float af[8];     // the weights rounded to FP32 (the FP32 solve: no FP64 conversion on the GPU)
};
enum { FACE_DROPPED = 1 };

// The chunked face solve.  The table is ordered along the line (it is built
// column by column, or row by row for steep lines).  Chunk c owns the
// entries [own_lo, own_hi); its items are the owned entries and every entry
// they depend on through the coupled corners, transitively (all within a few
// spacings along the line), sorted by level: an entry's level is 0 if no
// corner but its own site is a table entry, else one more than the highest
// level among those corners.  Every coupled corner lies strictly farther
// from the line than its point, so the levels are finite and a pass level
// by level, each level reading only lower ones, solves the system exactly.
// An item carries a copy of its entry's record (so that the solve's gather
// reads the item, then the corners' values: no dependent load of the table
// between them), the entry's index f, and kl[k]: the item index (within the
// chunk) of corner k, or -1 when corner k is not a table entry (or has
// weight 0).
constexpr int kFaceChunk = 256;      // entries a CTA owns
constexpr int kFaceLevels = 64;      // deepest coupling the chunked solve takes
constexpr int kFaceItemsMax = 1024;  // items a CTA holds in shared memory (a thread each)
struct FaceItem {
    LineFace rec;
    int32_t f;
    int16_t kl[8];
    int32_t pad;
};
struct FaceChunk {
    int32_t off, n, own_lo, own_hi;
    int32_t lv[kFaceLevels + 1];     // items of level L: [lv[L], lv[L + 1])
    int32_t pad[3];
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
template <typename T, typename D>
cudaError_t launch_line_faces_chunked(const StepArgs<T, D> &a, const FaceChunk *chunks, int n_chunks,
                                      const FaceItem *items, cudaStream_t s);

}  // namespace lbm
