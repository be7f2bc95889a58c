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
#include <cstdint>

#include "mfg_internal.cuh"
#include "reduce.cuh"

namespace mfg {

#define GRID_STRIDE(e, n) \
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (n); e += (long long)gridDim.x * blockDim.x)

// The vector kernels walk the data in pairs of doubles and use 16-byte accesses
// when every operand is 16-byte aligned (twice the bytes in flight per
// thread), single doubles otherwise.  Both paths visit the elements in the same
// order, so results do not depend on alignment (a batched instance at an odd
// offset gives the same bits as the same instance alone).
__device__ __forceinline__ bool aligned16(const void* a, const void* b = nullptr, const void* c = nullptr,
                                          const void* d = nullptr) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c) |
           reinterpret_cast<uintptr_t>(d)) & 15) == 0;
}

#define PAIR_LOOP(n, BODY2, BODY1, vec)                                                          \
  {                                                                                              \
    const long long n2_ = (n) >> 1;                                                              \
    _Pragma("unroll 4")                                                                          \
    for (long long e2 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e2 < n2_;              \
         e2 += (long long)gridDim.x * blockDim.x) {                                              \
      if (vec) {                                                                                 \
        BODY2                                                                                    \
      } else {                                                                                   \
        { const long long e = 2 * e2; BODY1 }                                                    \
        { const long long e = 2 * e2 + 1; BODY1 }                                                \
      }                                                                                          \
    }                                                                                            \
    if (((n) & 1) && blockIdx.x == 0 && threadIdx.x == 0) { const long long e = (n) - 1; BODY1 } \
  }

// p = zp, rz = r.zp (start of a solve, after the first preconditioner apply).
__global__ void __launch_bounds__(kThreads) k_init_p(long long n, const double* __restrict__ zp,
                                                     double* __restrict__ p, const double* __restrict__ r,
                                                     double* partials, DevScalars* sc) {
  if (sc->cg_done) return;
  double acc = 0.0;
  const bool vec = aligned16(zp, p, r);
  PAIR_LOOP(n, {
    const double2 v = reinterpret_cast<const double2*>(zp)[e2];
    reinterpret_cast<double2*>(p)[e2] = v;
    const double2 rv = reinterpret_cast<const double2*>(r)[e2];
    acc = fma(rv.x, v.x, acc);
    acc = fma(rv.y, v.y, acc);
  }, {
    const double v = zp[e];
    p[e] = v;
    acc = fma(r[e], v, acc);
  }, vec)
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
  const bool vec = aligned16(z, r, p, q);
  PAIR_LOOP(n, {
    double2 zv = reinterpret_cast<double2*>(z)[e2];
    const double2 pv = reinterpret_cast<const double2*>(p)[e2];
    double2 rv = reinterpret_cast<double2*>(r)[e2];
    const double2 qv = reinterpret_cast<const double2*>(q)[e2];
    zv.x = fma(alpha, pv.x, zv.x);
    zv.y = fma(alpha, pv.y, zv.y);
    rv.x = fma(-alpha, qv.x, rv.x);
    rv.y = fma(-alpha, qv.y, rv.y);
    reinterpret_cast<double2*>(z)[e2] = zv;
    reinterpret_cast<double2*>(r)[e2] = rv;
    acc = fma(rv.x, rv.x, acc);
    acc = fma(rv.y, rv.y, acc);
  }, {
    z[e] = fma(alpha, p[e], z[e]);
    const double rv = fma(-alpha, q[e], r[e]);
    r[e] = rv;
    acc = fma(rv, rv, acc);
  }, vec)
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
  const bool vec = aligned16(r, zp, q);
  PAIR_LOOP(n, {
    const double2 zv = reinterpret_cast<const double2*>(zp)[e2];
    const double2 rv = reinterpret_cast<const double2*>(r)[e2];
    a0 = fma(rv.x, zv.x, a0);
    a0 = fma(rv.y, zv.y, a0);
    if (FLEX) {
      const double2 qv = reinterpret_cast<const double2*>(q)[e2];
      a1 = fma(qv.x, zv.x, a1);
      a1 = fma(qv.y, zv.y, a1);
    }
  }, {
    const double zv = zp[e];
    a0 = fma(r[e], zv, a0);
    if (FLEX) a1 = fma(q[e], zv, a1);
  }, vec)
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
  const bool vec = aligned16(zp, p);
  PAIR_LOOP(n, {
    const double2 zv = reinterpret_cast<const double2*>(zp)[e2];
    double2 pv = reinterpret_cast<double2*>(p)[e2];
    pv.x = fma(beta, pv.x, zv.x);
    pv.y = fma(beta, pv.y, zv.y);
    reinterpret_cast<double2*>(p)[e2] = pv;
  }, { p[e] = fma(beta, p[e], zp[e]); }, vec)
}

void launch_init_p(long long n, const double* zp, double* p, const double* r, double* partials,
                   DevScalars* sc, cudaStream_t s, int cap) {
  k_init_p<<<red_blocks(n, cap), kThreads, 0, s>>>(n, zp, p, r, partials, sc);
}
void launch_update_zr(long long n, double* z, double* r, const double* p, const double* q,
                      double* partials, DevScalars* sc, cudaStream_t s, int cap) {
  k_update_zr<<<red_blocks(n, cap), kThreads, 0, s>>>(n, z, r, p, q, partials, sc);
}
void launch_dot_beta(long long n, const double* r, const double* zp, const double* q, int flexible,
                     double* partials, DevScalars* sc, cudaStream_t s, int cap) {
  if (flexible)
    k_dot_beta<1><<<red_blocks(n, cap), kThreads, 0, s>>>(n, r, zp, q, partials, sc);
  else
    k_dot_beta<0><<<red_blocks(n, cap), kThreads, 0, s>>>(n, r, zp, q, partials, sc);
}
void launch_update_p(long long n, const double* zp, double* p, DevScalars* sc,
                     cudaGraphConditionalHandle h, int use_handle, cudaStream_t s, int cap) {
  k_update_p<<<red_blocks(n, cap), kThreads, 0, s>>>(n, zp, p, sc, h, use_handle);
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
