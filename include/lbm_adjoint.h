/*
 * lbm_adjoint.h -- gradients of a sensor misfit through the time steps of
 * lbm.h, by the adjoint (transposed) time step.
 *
 * The paper (arXiv 2206.12412) defines only the forward method: the time
 * step of Sec. 3 with the boundary rules of Sec. 3.1 and the crack step of
 * Alg. 1 (Sec. 4.1).  This part differentiates it.  With the crack's cut
 * schedule held at the one the forward run took (the crack decisions of
 * Alg. 1 are discrete), one time step is affine in the state (w, wdot) and in
 * the Dirichlet edge values w*(t_n), so the gradient of
 *     L = sum_{n=1..T} sum_k (w^n(x_k) - wbar^n_k)^2
 * over a run of T steps is obtained exactly by running the transposed steps
 * in reverse order.  The transposed step is the same five-point update with
 * zero Dirichlet values plus a column-local correction at the crack-face
 * points (macroscopic rule of Sec. 3.1), so it needs no forward fields: only
 * the cut schedule (one int32 per step) and the sensor misfits (T x n_sens
 * FP64) recorded by the forward run.  Loss and gradient sums are FP64; the
 * adjoint fields use the handle's arithmetic (FP64 or FP32).
 *
 * A tape belongs to one handle.  lbm_tape_forward runs T steps of the
 * handle from its current state while recording; lbm_tape_backward then
 * produces dL/dw*_e(t_n) for the four edges and dL/dw0, dL/dwdot0 of the
 * state the forward run started from.  With checkpoint_every = k > 0 the
 * forward run keeps a snapshot of the handle's state every k steps instead
 * of the misfits of all T steps, and the backward sweep recomputes each
 * k-step segment from its snapshot before running its transposed steps
 * (about sqrt(T) snapshots for k = sqrt(T)); both forms give bit-identical
 * results.  Conventions (status codes, streams, sticky errors, allocator) are
 * those of lbm.h.
 */
#ifndef LBM_ADJOINT_H
#define LBM_ADJOINT_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_tape lbm_tape;

/* Make a tape for handle h (LBM_F64 or LBM_F32 storage; any crack mode -- a
 * K-criterion crack's decisions are those of the recorded run, and the
 * gradient is that of the run with this schedule).  sensors: 2 * n_sens
 * int32 in host memory, the (i, j) site of each sensor, 0 <= i < nx,
 * 0 <= j < ny (repeats allowed).  n_steps = T >= 1.
 * checkpoint_every: 0 keeps all misfits; k > 0 keeps ceil(T / k) + 1 state
 * snapshots instead.  allocator as in lbm_create (NULL: cudaMalloc).  The
 * tape holds device memory for T * n_sens misfits (k rows of them with
 * checkpoints), the snapshots, three adjoint planes and T * 4 * max(column
 * blocks, bands) partial sums.  The handle must outlive the tape and keep its
 * launch shape (lbm_set_launch) while the tape is used.  LBM_ERR_ARG for bad
 * input. */
lbm_status lbm_tape_create(lbm_handle *h, const int32_t *sensors, int32_t n_sens, int64_t n_steps,
                           int32_t checkpoint_every, const lbm_allocator *allocator, lbm_tape **out);

/* Run T steps of the handle from its current state (as lbm_step would) while
 * recording the cut schedule and the misfits r^n_k = w^n(x_k) - wbar^n_k
 * against targets (T x n_sens FP64, row n-1 for the state after step n, in
 * device memory if targets_on_device, else host memory).  The handle ends T
 * steps on.  If loss is not NULL it receives L in host memory (this
 * synchronises the stream); the loss also stays on the device for
 * lbm_tape_loss_device.  Any earlier recording of the tape is replaced. */
lbm_status lbm_tape_forward(lbm_tape *t, const double *targets, int32_t targets_on_device, double *loss);

/* Device pointer to L of the last lbm_tape_forward (FP64, valid until the
 * tape is destroyed; written on the handle's stream). */
lbm_status lbm_tape_loss_device(const lbm_tape *t, const double **loss);

/* The transposed sweep of the last recording.  Outputs (any may be NULL):
 *   dL_dload: 4 x T FP64, row e (LBM_LEFT .. LBM_TOP) holds dL/dw*_e(t_{n0+n})
 *             for the step n of the run (n0 the handle's step count when the
 *             forward run began); zero rows for non-Dirichlet edges.  In
 *             device memory if load_on_device.
 *   dL_dw0, dL_dwdot0: dense ny x nx arrays of dtype (LBM_F64 for F64
 *             storage, LBM_F32 for F32), the gradient with respect to the
 *             state the forward run started from; in device memory if
 *             fields_on_device.
 * With checkpoints the handle's state is recomputed segment by segment and
 * restored to the end of the forward run afterwards.  Returns LBM_ERR_STATE
 * without a recording, or if the handle's launch shape or loads changed since
 * the recording.  Host destinations synchronise the stream. */
lbm_status lbm_tape_backward(lbm_tape *t, double *dL_dload, int32_t load_on_device, void *dL_dw0, void *dL_dwdot0,
                             int32_t fields_on_device, int32_t dtype);

/* The misfits r^n_k (T x n_sens FP64) of the last recording, into host memory
 * (synchronises) or device memory.  LBM_ERR_STATE with checkpoints (only the
 * last segment's misfits are kept) or without a recording. */
lbm_status lbm_tape_misfits(lbm_tape *t, double *dst, int32_t dst_on_device);

/* Release the tape (NULL is ignored); synchronises the handle's stream. */
void lbm_tape_destroy(lbm_tape *t);

/* The whole sensor-misfit gradient in one call: lbm_tape_create(h, sensors,
 * n_sens, n_steps, checkpoint_every, allocator), lbm_tape_forward(targets,
 * targets_on_device, loss), lbm_tape_backward(dL_dload, load_on_device,
 * dL_dw0, dL_dwdot0, fields_on_device, dtype), lbm_tape_destroy -- the same
 * arguments, meanings and results (bit-identical to that sequence).  The
 * handle ends n_steps on, as after lbm_tape_forward; the stream is
 * synchronised before returning, so every output is complete.  The error of
 * the first call that fails is returned and the tape is released. */
lbm_status lbm_adjoint(lbm_handle *h, const int32_t *sensors, int32_t n_sens, int64_t n_steps, int32_t checkpoint_every,
                       const double *targets, int32_t targets_on_device, double *loss, double *dL_dload,
                       int32_t load_on_device, void *dL_dw0, void *dL_dwdot0, int32_t fields_on_device, int32_t dtype,
                       const lbm_allocator *allocator);

#ifdef __cplusplus
}
#endif

#endif /* LBM_ADJOINT_H */
