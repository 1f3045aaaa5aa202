/*
 * unet.h -- C ABI of the learned initial guess: a small 3D U-Net that predicts,
 * from a refinement level's density and its potential interpolated from the
 * parent (the initial guess of Sec. 2.4), the correction that brings that guess
 * closer to the level's solution, so that the multigrid iteration of Sec. 2.3
 * starts nearer its fixed point.  The paper has no learned component; this is
 * an addition, and the solver's stopping rule still decides convergence (a poor
 * prediction costs cycles, never accuracy).
 *
 * Network: 4 scales (edges n, n/2, n/4, n/8; n a power of two >= 8), widths
 * 16/32/64/64, 3x3x3 convolutions with bias and ReLU, 2x2x2 mean pooling,
 * nearest upsampling with concatenated skips, a 1x1x1 output; 367k FP32 master
 * parameters, BF16 tensor-core convolutions with FP32 accumulation.
 * Inputs per sample, on Omega (n^3, C order, x fastest):
 *   rho, phi_interp (FP64), resid = h^2 (4 pi G rho - lap_h(phi_interp)) (the
 *   7-point residual of the interpolated potential, scaled by h^2) and
 *   frho = 4 pi G h^2.
 * With s = max |phi_interp| and s_r = max |resid| the network sees
 * (frho * rho / s, phi_interp / s, resid / s_r) and predicts y; the guess is
 * phi_interp + (s_r n^2 / 16) y (the inverse Laplacian amplifies smooth
 * residuals by about n^2; the factor keeps y of order one for every n).
 * All array pointers are device pointers unless stated.  Return values: 0 ok,
 * 1 bad argument, 2 out of memory, 3 CUDA error, 4 a convolution's bounded
 * wait for its tensor-core work ran out (mg_unet_forward, mg_unet_train_step;
 * results invalid, the network keeps answering 4).  The convolutions run on
 * the 5th-generation tensor cores (tcgen05, accumulators in tensor memory). */
#ifndef MG_UNET_H
#define MG_UNET_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_unet mg_unet;

/* Number of FP32 parameters (all convolutions, then the 1x1 output). */
long mg_unet_param_count(void);

/* Allocate a network for up to bmax samples of edge up to nmax (power of
 * two); parameters initialised from seed (uniform, fan-in scaled).  stream:
 * cudaStream_t for every launch (NULL = legacy default stream). */
int mg_unet_create(int nmax, int bmax, unsigned long long seed, void *stream, mg_unet **out);
int mg_unet_destroy(mg_unet *u);

/* Parameters / gradient of the last training step as FP32 host arrays of
 * mg_unet_param_count() entries. */
int mg_unet_get_params(mg_unet *u, float *host_out);
int mg_unet_set_params(mg_unet *u, const float *host_in);
int mg_unet_get_grad(mg_unet *u, float *host_out);

/* Forward pass on B dense samples: y_out (host, may be NULL) receives
 * B * n^3 network outputs.  frho: host array of B factors. */
int mg_unet_forward(mg_unet *u, int B, int n, const double *rho, const double *phi_interp, const double *resid,
                    const double *frho, float *y_out);

/* One training step: loss = mean over the B * n^3 cells of
 * (y - (phi_true - phi_interp) / (s_r n^2 / 16))^2, backward pass into the parameter
 * gradient and, if update, one AdamW step (lr, decoupled weight decay wd).
 * loss_out (host) receives the loss before the update. */
int mg_unet_train_step(mg_unet *u, int B, int n, const double *rho, const double *phi_interp,
                       const double *resid, const double *phi_true, const double *frho, float lr, float wd, int update,
                       float *loss_out);

/* Convert the FP32 parameters into the BF16 copies the convolutions read
 * (done lazily otherwise); call before a solve graph records inference. */
int mg_unet_pack(mg_unet *u);

/* Solver hook: predict for B samples laid out as (n+4)^3 level blocks
 * (blk = 1, Omega at storage indices 2..n+1; the residual is formed from the
 * blocks, resid unused) or dense n^3 arrays (blk = 0, resid given), frho_dev a
 * device array of B factors, and (apply = 1) add the correction to phi on
 * Omega, all on `stream`. */
int mg_unet_predict_dev(mg_unet *u, int B, int n, int blk, const double *rho, double *phi, const double *resid,
                        const double *frho_dev, int apply, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MG_UNET_H */
