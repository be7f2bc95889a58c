// Vector kernels of the preconditioned CG solve with AAt (Sec. 3, the solve
// inside eq. CC*).  Every dot product is fused into the vector update that
// produces its operands; the last block turns the partial sums into the CG
// scalars, so no scalar ever travels to the host.
//
// Solve:  AAt delta = sigma (C ybar - d)  with z <- z + delta in place, i.e.
// the PCG iterate is z itself started from z_l (the residual of z_l for the
// system of eq. CC* is exactly sigma (C ybar - d) when x_l = C^T z_l).
//
// Iteration (Fletcher-Reeves; Polak-Ribiere "flexible" when P^{-1} is FP32):
//   q = AAt p; alpha = rz/(p.q); z += alpha p; r -= alpha q;
//   stop if ||r|| <= tol ||r_0||;  zp = P^{-1} r;
//   beta = (r.zp)/rz (FR)  or  -alpha (q.zp)/rz (PR);  rz = r.zp;  p = zp + beta p.
#include "mfg_internal.cuh"
#include "reduce.cuh"

namespace mfg {

#define GRID_STRIDE(e, n) \
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (n); e += (long long)gridDim.x * blockDim.x)

// p = zp, rz = r.zp (start of a solve, after the first preconditioner apply).
__global__ void __launch_bounds__(kThreads) k_init_p(long long n, const double* __restrict__ zp,
                                                     double* __restrict__ p, const double* __restrict__ r,
                                                     double* partials, DevScalars* sc) {
  if (sc->cg_done) return;
  double acc = 0.0;
  GRID_STRIDE(e, n) {
    const double v = zp[e];
    p[e] = v;
    acc += r[e] * v;
  }
  double part[1] = {acc};
  block_sum<1>(part);
  if (!publish_and_check_last<1>(part, partials, &sc->counter)) return;
  double tot[1];
  gather_partials<1>(partials, tot);
  if (flat_tid() == 0) {
    sc->rz = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      // r.P^{-1}r must be positive for r != 0 (P is SPD).
      sc->cg_done = 1;
      if (sc->status == MFG_OK) sc->status = MFG_ERR_NONFINITE;
    }
    sc->counter = 0;
  }
}

// z += alpha p; r -= alpha q; rr = r.r; convergence test.
__global__ void __launch_bounds__(kThreads) k_update_zr(long long n, double* __restrict__ z,
                                                        double* __restrict__ r, const double* __restrict__ p,
                                                        const double* __restrict__ q, double* partials,
                                                        DevScalars* sc) {
  if (sc->cg_done) return;
  const double alpha = sc->alpha;
  double acc = 0.0;
  GRID_STRIDE(e, n) {
    z[e] += alpha * p[e];
    const double rv = r[e] - alpha * q[e];
    r[e] = rv;
    acc += rv * rv;
  }
  double part[1] = {acc};
  block_sum<1>(part);
  if (!publish_and_check_last<1>(part, partials, &sc->counter)) return;
  double tot[1];
  gather_partials<1>(partials, tot);
  if (flat_tid() == 0) {
    sc->rr = tot[0];
    sc->cg_it += 1;
    const double tol = sc->cg_tol;
    if (!isfinite(tot[0])) {
      sc->cg_done = 1;
      if (sc->status == MFG_OK) sc->status = MFG_ERR_NONFINITE;
    } else if (tot[0] <= tol * tol * sc->bnorm2) {
      sc->cg_done = 1;
    } else if (sc->cg_it >= sc->max_cg) {
      sc->cg_done = 1;
      if (sc->status == MFG_OK) sc->status = MFG_ERR_NOT_CONVERGED;
    }
    sc->counter = 0;
  }
}

// rz_new = r.zp (and qz = q.zp for the flexible variant); beta; rz = rz_new.
template <int FLEX>
__global__ void __launch_bounds__(kThreads) k_dot_beta(long long n, const double* __restrict__ r,
                                                       const double* __restrict__ zp,
                                                       const double* __restrict__ q, double* partials,
                                                       DevScalars* sc) {
  if (sc->cg_done) return;
  double a0 = 0.0, a1 = 0.0;
  GRID_STRIDE(e, n) {
    const double zv = zp[e];
    a0 += r[e] * zv;
    if (FLEX) a1 += q[e] * zv;
  }
  double part[2] = {a0, a1};
  block_sum<2>(part);
  if (!publish_and_check_last<2>(part, partials, &sc->counter)) return;
  double tot[2];
  gather_partials<2>(partials, tot);
  if (flat_tid() == 0) {
    const double rz_old = sc->rz;
    sc->qz = tot[1];
    sc->beta = FLEX ? (-sc->alpha * tot[1] / rz_old) : (tot[0] / rz_old);
    sc->rz = tot[0];
    if (!isfinite(sc->beta) || !(tot[0] > 0.0)) {
      sc->cg_done = 1;
      if (sc->status == MFG_OK) sc->status = MFG_ERR_NONFINITE;
    }
    sc->counter = 0;
  }
}

// p = zp + beta p; ends the CG body: keeps the while-node running until done.
__global__ void __launch_bounds__(kThreads) k_update_p(long long n, const double* __restrict__ zp,
                                                       double* __restrict__ p, DevScalars* sc,
                                                       cudaGraphConditionalHandle h, int use_handle) {
  const int done = sc->cg_done;
  if (use_handle && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, done ? 0u : 1u);
  if (done) return;
  const double beta = sc->beta;
  GRID_STRIDE(e, n) { p[e] = zp[e] + beta * p[e]; }
}

void launch_init_p(long long n, const double* zp, double* p, const double* r, double* partials,
                   DevScalars* sc, cudaStream_t s) {
  k_init_p<<<red_blocks(n), kThreads, 0, s>>>(n, zp, p, r, partials, sc);
}
void launch_update_zr(long long n, double* z, double* r, const double* p, const double* q,
                      double* partials, DevScalars* sc, cudaStream_t s) {
  k_update_zr<<<red_blocks(n), kThreads, 0, s>>>(n, z, r, p, q, partials, sc);
}
void launch_dot_beta(long long n, const double* r, const double* zp, const double* q, int flexible,
                     double* partials, DevScalars* sc, cudaStream_t s) {
  if (flexible)
    k_dot_beta<1><<<red_blocks(n), kThreads, 0, s>>>(n, r, zp, q, partials, sc);
  else
    k_dot_beta<0><<<red_blocks(n), kThreads, 0, s>>>(n, r, zp, q, partials, sc);
}
void launch_update_p(long long n, const double* zp, double* p, DevScalars* sc,
                     cudaGraphConditionalHandle h, int use_handle, cudaStream_t s) {
  k_update_p<<<red_blocks(n), kThreads, 0, s>>>(n, zp, p, sc, h, use_handle);
}

// Start of a CP iteration inside the graph: arms the inner while-node.
__global__ void k_scalars_begin(DevScalars* sc, cudaGraphConditionalHandle h, int use_handle) {
  if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(h, sc->cg_done ? 0u : 1u);
}
void launch_scalars_begin(DevScalars* sc, cudaGraphConditionalHandle h, int use_handle,
                          cudaStream_t s) {
  k_scalars_begin<<<1, 32, 0, s>>>(sc, h, use_handle);
}

}  // namespace mfg
