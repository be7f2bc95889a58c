// Per-cell proximal map of tau*phi (Sec. 3), fused with the dual lift
// x = C^T z, the primal step y - tau x, the extrapolation
// ybar = y_new + theta (y_new - y) and the step-size update of Sec. 5.
//
// The paper takes prox_{tau phi_ij} from its reference (BAKS, Cor. 3.1) without
// printing it.  For q' = 2 the first-order conditions give, with
// P = P_K(w_bar) (projection onto the cone K of Sec. 2):
//   w = m/(m + tau) P,
//   h(m) = m - m_bar + tau f_eff(m) - tau |P|^2 / (2 (m + tau)^2) = 0,
// h strictly increasing (f_eff nondecreasing); m = 0, w = 0 when h(0) >= 0,
// otherwise the root lies in (0, m_hi], m_hi = max(0, m_bar - tau f_eff(0)) +
// |P|^2/(2 tau).  f_eff(m) = f_a m + f_b m^2 + V(x), plus (g_a m + W(x))/dt on
// the last plane (G weighted by 1/dt in calF, Sec. 2).
//
// Root finder: Newton from m = 0 with the bracket [lo, hi] kept by the sign of
// h and a bisection step whenever Newton leaves it (for f_b = 0, h is concave
// and Newton from the left never does); see prox_cell for the precision split.
#include "mfg_internal.cuh"
#include "reduce.cuh"

namespace mfg {

// 1/d in FP64 without the FP64 divide: an FP32 reciprocal seed refined by two
// Newton-Raphson steps r <- r (2 - d r) (the classical reciprocal iteration;
// each step squares the relative error, 1e-7 -> 1e-14 -> round-off).  Valid
// for d in the FP32 normal range, which the callers check.
__device__ __forceinline__ double rcp64(double d) {
  double r = (double)(1.0f / (float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

// Safeguarded Newton on h in FP32, from x = 0 with the bracket [0, hi].
__device__ __forceinline__ float newton_h32(float hi, float B, float hP, float tau, float a1, float tb) {
  float x = 0.0f, lo = 0.0f;
  for (int it = 0; it < 24; ++it) {
    const float it1 = 1.0f / (x + tau);
    const float it2 = it1 * it1;
    const float hx = fmaf(tb, x * x, a1 * x) - B - hP * it2;
    if (hx < 0.0f) lo = x; else hi = x;
    if (hx == 0.0f) break;
    const float dh = fmaf(2.0f * tb, x, a1) + 2.0f * hP * it2 * it1;
    float xn = x - hx / dh;
    if (!(xn >= lo && xn <= hi)) xn = 0.5f * (lo + hi);
    const float dxv = fabsf(xn - x);
    x = xn;
    if (dxv <= 2e-7f * x || hi - lo <= 2e-7f * hi) break;
  }
  return x;
}

// Root of h(m) = (1 + tau a) m + tau b m^2 - B - hP/(m + tau)^2 with
// B = m_bar - tau c and hP = tau |P|^2 / 2 (the scalar equation above, with
// the FP64 constants combined before any rounding to FP32).  FP64 runs at
// about 1/58 of the FP32 rate on GB300, so the iteration runs in FP32 and FP64
// Newton steps polish the result; the polish stops once a step is below
// 1e-8 relative (quadratic convergence leaves ~1e-16) and keeps the bracket,
// bisecting if a step leaves it.
template <int NW>
__device__ __forceinline__ void prox_cell(double mbar, const double (&wbar)[NW], double tau,
                                          double inv_tau, double a, double b, double c, double& m,
                                          double (&w)[NW]) {
  // projection onto K by sign tests on the bit patterns (no FP64 min/max)
  double P[NW];
  double P2 = 0.0;
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const bool neg = __double_as_longlong(wbar[q]) < 0;
    P[q] = ((q & 1) ? neg : !neg) ? wbar[q] : 0.0;
    P2 = fma(P[q], P[q], P2);
  }
  const double B = mbar - tau * c;
  const double half_P2_tau = 0.5 * P2 * inv_tau;
  if (-B - half_P2_tau >= 0.0) {  // h(0) >= 0
    m = 0.0;
#pragma unroll
    for (int q = 0; q < NW; ++q) w[q] = 0.0;
    return;
  }
  double hi = (B > 0.0 ? B : 0.0) + half_P2_tau;
  double lo = 0.0;
  const double hP = 0.5 * tau * P2;
  const double a1 = fma(tau, a, 1.0), tb = tau * b;
  const bool fp32_ok = hi < 1e30 && hP < 1e30 && fabs(B) < 1e30 && tau > 1e-30 && tau < 1e30;
  double x = 0.0;
  // FP64 polish: from an FP32 root (relative error ~1e-7) one Newton step
  // leaves ~1e-14; another step is taken only if the first moved by more than
  // 2e-7 relative (an FP32 root spoiled by cancellation) or there was no FP32 root.
  double stop = 2e-7;
  if (fp32_ok) {
    x = (double)newton_h32((float)hi, (float)B, (float)hP, (float)tau, (float)a1, (float)tb);
  } else {
    stop = 1e-8;
  }
  for (int it = 0; it < 100; ++it) {
    const double t = x + tau;
    const double it1 = fp32_ok ? rcp64(t) : 1.0 / t;
    const double it2 = it1 * it1;
    const double hx = fma(tb, x * x, a1 * x) - B - hP * it2;
    if (hx < 0.0) lo = x; else hi = x;
    if (hx == 0.0) break;
    const double dh = fma(2.0 * tb, x, a1) + 2.0 * hP * it2 * it1;
    double xn = x - hx * ((fp32_ok && dh < 1e37) ? rcp64(dh) : 1.0 / dh);
    if (!(xn >= lo && xn <= hi)) xn = 0.5 * (lo + hi);
    const double dxv = fabs(xn - x);
    x = xn;
    if (dxv <= stop * x || hi - lo <= 4e-16 * hi) break;
    stop = 1e-8;
  }
  m = x;
  const double s = x * (fp32_ok ? rcp64(x + tau) : 1.0 / (x + tau));
#pragma unroll
  for (int q = 0; q < NW; ++q) w[q] = s * P[q];
}

// y, ybar hold c planes; z one plane set.  Cell e pairs (m^{k+1}, w^k).
template <int ACTX>
__global__ void __launch_bounds__(kThreads) k_prox_cp(Geom g, Coef cf, const double* __restrict__ z,
                                                      double* __restrict__ y, double* __restrict__ ybar,
                                                      const double* __restrict__ V,
                                                      const double* __restrict__ W, double* partials,
                                                      DevScalars* sc, cudaGraphConditionalHandle h,
                                                      int use_handle) {
  constexpr int NW = ACTX ? 4 : 2;
  const long long n = g.n;
  const double tau = sc->tau;
  const double inv_tau = 1.0 / tau;
  const double theta = 1.0 / sqrt(1.0 + 2.0 * cf.gamma * tau);
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.ny);
    const long long t = e / g.ny;
    const int i = (int)(t % g.nx);
    const int k = (int)(t / g.nx);
    const long long base = (long long)k * g.S;
    const long long rowi = base + (long long)i * g.ny;
    // x = C^T z at this cell
    const double zc = z[e];
    const bool per_y = g.pery;
    const bool hmy = per_y || j >= 1, hpy = per_y || j <= g.ny - 2;
    const int jm = hmy ? (j == 0 ? g.ny - 1 : j - 1) : j;
    const int jp = hpy ? (j == g.ny - 1 ? 0 : j + 1) : j;
    const double zjm = z[rowi + jm], zjp = z[rowi + jp];
    // K z: cK z - ay (zN + zS) - ax (zW + zE) away from Neumann ends (fewer FP64 ops)
    double Kz;
    double xw[NW];
    if (ACTX) {
      const bool per_x = g.perx;
      const bool hmx = per_x || i >= 1, hpx = per_x || i <= g.nx - 2;
      const int im = hmx ? (i == 0 ? g.nx - 1 : i - 1) : i;
      const int ip = hpx ? (i == g.nx - 1 ? 0 : i + 1) : i;
      const double zim = z[base + (long long)im * g.ny + j], zip = z[base + (long long)ip * g.ny + j];
      if (hmx && hpx && hmy && hpy)
        Kz = fma(2.0 * (g.ax + g.ay), zc, -fma(g.ax, zim + zip, g.ay * (zjm + zjp)));
      else
        Kz = g.ay * ((hmy ? zc - zjm : 0.0) + (hpy ? zc - zjp : 0.0)) +
             g.ax * ((hmx ? zc - zim : 0.0) + (hpx ? zc - zip : 0.0));
      xw[0] = hpx ? (zc - zip) * g.idx : 0.0;
      xw[1] = hmx ? (zim - zc) * g.idx : 0.0;
      xw[2] = hpy ? (zc - zjp) * g.idy : 0.0;
      xw[3] = hmy ? (zjm - zc) * g.idy : 0.0;
    } else {
      Kz = g.ay * ((hmy ? zc - zjm : 0.0) + (hpy ? zc - zjp : 0.0));
      xw[0] = hpy ? (zc - zjp) * g.idy : 0.0;
      xw[1] = hmy ? (zjm - zc) * g.idy : 0.0;
    }
    const double zn = (k + 1 < g.nt) ? z[e + g.S] : 0.0;
    const double xm = fma(g.nu, Kz, (zc - zn) * g.idt);
    // prox of y - tau x
    const double m_old = y[e];
    double w_old[NW], wbar[NW], w_new[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      w_old[q] = y[e + (q + 1) * n];
      wbar[q] = w_old[q] - tau * xw[q];
    }
    const bool last = (k == g.nt - 1);
    const long long f = (long long)i * g.ny + j;
    const double a = cf.f_a + (last ? cf.g_a * g.idt : 0.0);
    const double cc = V[f] + (last ? W[f] * g.idt : 0.0);
    double m_new;
    prox_cell<NW>(m_old - tau * xm, wbar, tau, inv_tau, a, cf.f_b, cc, m_new, w_new);
    y[e] = m_new;
    ybar[e] = m_new + theta * (m_new - m_old);
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      y[e + (q + 1) * n] = w_new[q];
      ybar[e + (q + 1) * n] = w_new[q] + theta * (w_new[q] - w_old[q]);
    }
    const double dm = m_new - m_old;
    acc = fma(dm, dm, acc);
  }
  double part[1] = {acc};
  block_sum<1>(part);
  if (!publish_and_check_last<1>(part, partials, &sc->counter)) return;
  double tot[1];
  gather_partials<1>(partials, tot);
  if (flat_tid() == 0) {
    const double r = sqrt(tot[0]);
    sc->dm2 = tot[0];
    sc->r_last = r;
    sc->tau = theta * tau;
    sc->sigma = sc->sigma / theta;
    sc->ell += 1;
    sc->cp_iters += 1;
    sc->cg_total += sc->cg_it;
    if (sc->cg_it > sc->cg_max) sc->cg_max = sc->cg_it;
    sc->cp_left -= 1;
    if (!isfinite(r)) {
      sc->status = MFG_ERR_NONFINITE;
      sc->cp_done = 1;
    }
    if (sc->status == MFG_ERR_NONFINITE) sc->cp_done = 1;
    if (sc->cp_tol > 0.0 && r <= sc->cp_tol) sc->cp_done = 1;
    if (use_handle) cudaGraphSetConditional(h, (sc->cp_left > 0 && !sc->cp_done) ? 1u : 0u);
    sc->counter = 0;
  }
}

template <int ACTX>
__global__ void __launch_bounds__(kThreads) k_prox_plain(Geom g, Coef cf, double tau,
                                                         const double* v, double* y,
                                                         const double* __restrict__ V,
                                                         const double* __restrict__ W) {
  constexpr int NW = ACTX ? 4 : 2;
  const long long n = g.n;
  const double inv_tau = 1.0 / tau;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / g.S);
    const long long f = e % g.S;
    double wbar[NW], w_new[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) wbar[q] = v[e + (q + 1) * n];
    const bool last = (k == g.nt - 1);
    const double a = cf.f_a + (last ? cf.g_a * g.idt : 0.0);
    const double cc = V[f] + (last ? W[f] * g.idt : 0.0);
    double m_new;
    prox_cell<NW>(v[e], wbar, tau, inv_tau, a, cf.f_b, cc, m_new, w_new);
    y[e] = m_new;
#pragma unroll
    for (int q = 0; q < NW; ++q) y[e + (q + 1) * n] = w_new[q];
  }
}

void launch_prox_cp(const Geom& g, const Coef& cf, const double* z, double* y, double* ybar,
                    const double* V, const double* W, double* partials, DevScalars* sc,
                    cudaGraphConditionalHandle h, int use_handle, cudaStream_t s) {
  const int nb = red_blocks(g.n);
  if (g.actx)
    k_prox_cp<1><<<nb, kThreads, 0, s>>>(g, cf, z, y, ybar, V, W, partials, sc, h, use_handle);
  else
    k_prox_cp<0><<<nb, kThreads, 0, s>>>(g, cf, z, y, ybar, V, W, partials, sc, h, use_handle);
}

void launch_prox_plain(const Geom& g, const Coef& cf, double tau, const double* v, double* y,
                       const double* V, const double* W, cudaStream_t s) {
  const int nb = red_blocks(g.n);
  if (g.actx)
    k_prox_plain<1><<<nb, kThreads, 0, s>>>(g, cf, tau, v, y, V, W);
  else
    k_prox_plain<0><<<nb, kThreads, 0, s>>>(g, cf, tau, v, y, V, W);
}

}  // namespace mfg
