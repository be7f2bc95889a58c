// Adjoint of the converged equilibrium by implicit differentiation of the KKT
// conditions of (VMFG_h) (Sec. 2-3).  At a CP solution (y, z):
//   R1 = grad phi_A(y) + (C^T z)_A = 0   (active set A: m > 0, w_c != 0),
//   R2 = C y - d(m0) = 0.
// The adjoint system [[H, C_A^T], [C_A, 0]] [mu; eta] = [g; 0], with H the
// per-cell Hessian of phi = b_hat + F on A, is solved through its Schur
// complement (C_A H^{-1} C_A^T) eta = C_A H^{-1} g by the same PCG kernels
// and the same preconditioner P as the forward solve, then
// mu = H^{-1} (g - C^T eta).  Gradients (dloss/dtheta = -[mu; eta].dR/dtheta):
//   dm0(x) = eta(0, x)/dt,  dV(x) = -sum_k mu_m(k, x),  dW(x) = -mu_m(N_t-1, x)/dt,
//   dnu = -sum mu_m (K z) - sum eta (K m);
// with a viscosity field, K_nu in C and, per node a (dK_nu/dnu_a = sum over
// the faces f of a of g_f g_f^T / (2 dx^2), g_f the face difference),
//   dnu(a) = -(1/2) sum_k sum_{f of a} [(g_f.mu_m)(g_f.z) + (g_f.eta)(g_f.m)] / dx^2.
//
// H^{-1} per cell in closed form.  With a' = f_eff'(m) (f_a + 2 f_b m, plus
// g_a/dt on the last plane), H = [[|w|^2/m^3 + a', -w^T/m^2], [-w/m^2, I/m]]
// on the active components; its Schur complement in m is exactly a' because
// the inactive w components are zero, so
//   (H^{-1} u)_m = (u_m + w.u_w / m) / a',  (H^{-1} u)_w = m u_w + (w/m) (H^{-1} u)_m,
// and 0 on inactive components.
#include "mfg_internal.cuh"
#include "reduce.cuh"

namespace mfg {

template <int NW>
__device__ __forceinline__ void hinv_cell(double m, const double (&w)[NW], double ap, double um,
                                          const double (&uw)[NW], double& om, double (&ow)[NW]) {
  if (!(m > 0.0)) {
    om = 0.0;
#pragma unroll
    for (int q = 0; q < NW; ++q) ow[q] = 0.0;
    return;
  }
  const double im = 1.0 / m;
  double wu = 0.0;
#pragma unroll
  for (int q = 0; q < NW; ++q) wu = fma(w[q], uw[q], wu);
  om = (um + wu * im) / ap;
#pragma unroll
  for (int q = 0; q < NW; ++q) ow[q] = (w[q] != 0.0) ? fma(m, uw[q], w[q] * im * om) : 0.0;
}

template <int ACTX>
__device__ __forceinline__ void load_cell(const double* y, long long e, long long n, double& m,
                                          double (&w)[ACTX ? 4 : 2]) {
  m = y[e];
#pragma unroll
  for (int q = 0; q < (ACTX ? 4 : 2); ++q) w[q] = y[e + (q + 1) * n];
}

template <int ACTX>
__global__ void __launch_bounds__(kThreads) k_hinv(Geom g, Coef cf, const double* __restrict__ y,
                                                   const double* __restrict__ u, double* __restrict__ out) {
  constexpr int NW = ACTX ? 4 : 2;
  const long long n = g.n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / g.S);
    double m, w[NW], uw[NW], ow[NW], om;
    load_cell<ACTX>(y, e, n, m, w);
#pragma unroll
    for (int q = 0; q < NW; ++q) uw[q] = u[e + (q + 1) * n];
    const double ap = cf.f_a + 2.0 * cf.f_b * m + (k == g.nt - 1 ? cf.g_a * g.idt : 0.0);
    hinv_cell<NW>(m, w, ap, u[e], uw, om, ow);
    out[e] = om;
#pragma unroll
    for (int q = 0; q < NW; ++q) out[e + (q + 1) * n] = ow[q];
  }
}

// out = H^{-1} (C^T p)  or, with gsub, out = H^{-1} (gsub - C^T p).  VN: L =
// K_nu + I/dt with the face coefficients of Geom::kfx / kfy.
template <int ACTX, bool VN>
__global__ void __launch_bounds__(kThreads) k_ct_hinv(Geom g, Coef cf, const double* __restrict__ y,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ gsub,
                                                      double* __restrict__ out, const DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  constexpr int NW = ACTX ? 4 : 2;
  const long long n = g.n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.ny);
    const long long t = e / g.ny;
    const int i = (int)(t % g.nx);
    const int k = (int)(t / g.nx);
    const long long base = (long long)k * g.S;
    const long long rowi = base + (long long)i * g.ny;
    const double pc = p[e];
    const bool hmy = g.pery || j >= 1, hpy = g.pery || j <= g.ny - 2;
    const int jm = hmy ? (j == 0 ? g.ny - 1 : j - 1) : j;
    const int jp = hpy ? (j == g.ny - 1 ? 0 : j + 1) : j;
    const double pjm = p[rowi + jm], pjp = p[rowi + jp];
    const long long f0 = (long long)i * g.ny;
    // K_nu p: a missing face has its neighbour index at the node itself (difference 0)
    double Kp = VN ? fma(g.kfy[f0 + j], pc - pjp, g.kfy[f0 + jm] * (pc - pjm))
                   : g.ay * ((hmy ? pc - pjm : 0.0) + (hpy ? pc - pjp : 0.0));
    double xw[NW];
    if (ACTX) {
      const bool hmx = g.perx || i >= 1, hpx = g.perx || i <= g.nx - 2;
      const int im = hmx ? (i == 0 ? g.nx - 1 : i - 1) : i;
      const int ip = hpx ? (i == g.nx - 1 ? 0 : i + 1) : i;
      const double pim = p[base + (long long)im * g.ny + j], pip = p[base + (long long)ip * g.ny + j];
      if (VN)
        Kp = fma(g.kfx[f0 + j], pc - pip, fma(g.kfx[(long long)im * g.ny + j], pc - pim, Kp));
      else
        Kp += g.ax * ((hmx ? pc - pim : 0.0) + (hpx ? pc - pip : 0.0));
      xw[0] = hpx ? (pc - pip) * g.idx : 0.0;
      xw[1] = hmx ? (pim - pc) * g.idx : 0.0;
      xw[2] = hpy ? (pc - pjp) * g.idy : 0.0;
      xw[3] = hmy ? (pjm - pc) * g.idy : 0.0;
    } else {
      xw[0] = hpy ? (pc - pjp) * g.idy : 0.0;
      xw[1] = hmy ? (pjm - pc) * g.idy : 0.0;
    }
    const double pn = (k + 1 < g.nt) ? p[e + g.S] : 0.0;
    double xm = (VN ? Kp : g.nu * Kp) + (pc - pn) * g.idt;
    if (gsub != nullptr) {
      xm = gsub[e] - xm;
#pragma unroll
      for (int q = 0; q < NW; ++q) xw[q] = gsub[e + (q + 1) * n] - xw[q];
    }
    double m, w[NW], ow[NW], om;
    load_cell<ACTX>(y, e, n, m, w);
    const double ap = cf.f_a + 2.0 * cf.f_b * m + (k == g.nt - 1 ? cf.g_a * g.idt : 0.0);
    hinv_cell<NW>(m, w, ap, xm, xw, om, ow);
    out[e] = om;
#pragma unroll
    for (int q = 0; q < NW; ++q) out[e + (q + 1) * n] = ow[q];
  }
}

// One thread per spatial point, looping over time planes; dnu by reduction,
// or (VN) the node derivative dnu(f) written per point.
template <bool VN>
__global__ void __launch_bounds__(kThreads) k_adj_grads(Geom g, const double* __restrict__ y,
                                                        const double* __restrict__ z,
                                                        const double* __restrict__ eta,
                                                        const double* __restrict__ mu, double* dm0,
                                                        double* dV, double* dW, double* dnu,
                                                        double* partials, DevScalars* sc) {
  double acc = 0.0;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < g.S;
       f += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(f % g.ny), i = (int)(f / g.ny);
    const bool hmy = g.pery || j >= 1, hpy = g.pery || j <= g.ny - 2;
    const int jm = hmy ? (j == 0 ? g.ny - 1 : j - 1) : j;
    const int jp = hpy ? (j == g.ny - 1 ? 0 : j + 1) : j;
    const bool hmx = g.actx && (g.perx || i >= 1), hpx = g.actx && (g.perx || i <= g.nx - 2);
    const int im = hmx ? (i == 0 ? g.nx - 1 : i - 1) : i;
    const int ip = hpx ? (i == g.nx - 1 ? 0 : i + 1) : i;
    double sv = 0.0, node = 0.0;
    for (int k = 0; k < g.nt; ++k) {
      const long long base = (long long)k * g.S;
      const long long e = base + f;
      const double mum = mu[e];
      sv += mum;
      if (VN) {
        // the node's faces: (g.mu)(g.z) + (g.eta)(g.m) per face, times 1/dx^2
        auto face = [&](long long nb, double c) {
          const double a = (mum - mu[nb]) * (z[e] - z[nb]) + (eta[e] - eta[nb]) * (y[e] - y[nb]);
          return c * a;
        };
        double t = 0.0;
        if (hmy) t += face(base + (long long)i * g.ny + jm, g.ay);
        if (hpy) t += face(base + (long long)i * g.ny + jp, g.ay);
        if (hmx) t += face(base + (long long)im * g.ny + j, g.ax);
        if (hpx) t += face(base + (long long)ip * g.ny + j, g.ax);
        node += t;
      } else {
        auto K5 = [&](const double* a) {
          const double c = a[e];
          return g.ay * ((hmy ? c - a[base + (long long)i * g.ny + jm] : 0.0) +
                         (hpy ? c - a[base + (long long)i * g.ny + jp] : 0.0)) +
                 g.ax * ((hmx ? c - a[base + (long long)im * g.ny + j] : 0.0) +
                         (hpx ? c - a[base + (long long)ip * g.ny + j] : 0.0));
        };
        acc -= mum * K5(z) + eta[e] * K5(y);
      }
    }
    if (VN) dnu[f] = -0.5 * node;
    dm0[f] = eta[f] * g.idt;
    dV[f] = -sv;
    if (dW != nullptr) dW[f] = -mu[(long long)(g.nt - 1) * g.S + f] * g.idt;
  }
  if (VN) return;
  double part[1] = {acc};
  block_sum<1>(part);
  if (!publish_and_check_last<1>(part, partials, &sc->counter)) return;
  double tot[1];
  gather_partials<1>(partials, tot);
  if (flat_tid() == 0) {
    *dnu = tot[0];
    sc->counter = 0;
  }
}

void launch_hinv(const Geom& g, const Coef& cf, const double* y, const double* u, double* out,
                 cudaStream_t s) {
  const int nb = red_blocks(g.n, g.vec_blocks);
  if (g.actx)
    k_hinv<1><<<nb, kThreads, 0, s>>>(g, cf, y, u, out);
  else
    k_hinv<0><<<nb, kThreads, 0, s>>>(g, cf, y, u, out);
}

void launch_ct_hinv(const Geom& g, const Coef& cf, const double* y, const double* p,
                    const double* gsub, double* out, cudaStream_t s, const DevScalars* sc) {
  const int nb = red_blocks(g.n, g.vec_blocks);
  const bool vn = g.kfy != nullptr;
  if (g.actx && vn)
    k_ct_hinv<1, true><<<nb, kThreads, 0, s>>>(g, cf, y, p, gsub, out, sc);
  else if (g.actx)
    k_ct_hinv<1, false><<<nb, kThreads, 0, s>>>(g, cf, y, p, gsub, out, sc);
  else if (vn)
    k_ct_hinv<0, true><<<nb, kThreads, 0, s>>>(g, cf, y, p, gsub, out, sc);
  else
    k_ct_hinv<0, false><<<nb, kThreads, 0, s>>>(g, cf, y, p, gsub, out, sc);
}

void launch_adj_grads(const Geom& g, const double* y, const double* z, const double* eta,
                      const double* mu, double* dm0, double* dV, double* dW, double* dnu,
                      double* partials, DevScalars* sc, cudaStream_t s) {
  const int nb = red_blocks(g.S, g.vec_blocks);
  if (g.kfy != nullptr)
    k_adj_grads<true><<<nb, kThreads, 0, s>>>(g, y, z, eta, mu, dm0, dV, dW, dnu, partials, sc);
  else
    k_adj_grads<false><<<nb, kThreads, 0, s>>>(g, y, z, eta, mu, dm0, dV, dW, dnu, partials, sc);
}

}  // namespace mfg
