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
#include <algorithm>

#include "df64.cuh"
#include "mfg_internal.cuh"
#include "reduce.cuh"

namespace mfg {

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

// FP64 Newton on h from x = 0 with bisection safeguard: the path for inputs
// outside the FP32 range of the fast path.
// A NaN in the cell's data (m_bar, the fluxes, V, W or the dual) comes out as
// NaN rather than as a bracketed root, so the CP step norm reports it.
__device__ __noinline__ double newton_h64(double B, double hP, double tau, double a1, double tb, double hi) {
  if (isnan(B) || isnan(hP)) return __longlong_as_double(0x7ff8000000000000LL);
  double x = 0.0, lo = 0.0;
  for (int it = 0; it < 200; ++it) {
    const double it1 = 1.0 / (x + tau);
    const double it2 = it1 * it1;
    const double hx = fma(tb, x * x, a1 * x) - B - hP * it2;
    if (hx < 0.0) lo = x; else hi = x;
    if (hx == 0.0) break;
    const double dh = fma(2.0 * tb, x, a1) + 2.0 * hP * it2 * it1;
    double xn = x - hx / dh;
    if (!(xn >= lo && xn <= hi)) xn = 0.5 * (lo + hi);
    const double dxv = fabs(xn - x);
    x = xn;
    if (dxv <= 1e-16 * x || hi - lo <= 4e-16 * hi) break;
  }
  return x;
}

// Prox for the general power Hamiltonian |p|^{q'}/q', q = q'/(q'-1), b_hat =
// |w|^q/(q m^{q-1}) (Sec. 2).  For fixed m > 0 the minimising flux is
// w = m t P/|P| with t >= 0 the root of g(t) = m t + tau t^{q-1} - |P|, and m
// is the root of the increasing function
//   h_q(m) = a1 m + tau b m^2 - B - (tau/q') t(m)^q,
// h_q'(m) = a1 + 2 tau b m + tau (q-1) t^q / (m + tau (q-1) t^{q-2}),
// with (0, 0) the prox when h_q(0) = -B - (tau/q') (|P|/tau)^{q'} >= 0 and the
// root in (0, max(0, B) + (tau/q') (|P|/tau)^{q'}] otherwise.  Both roots by
// safeguarded Newton in FP64 (the bracket kept by the sign, a bisection step
// whenever Newton leaves it).  q' = 2 never takes this path.
__device__ double velocity_q(double m, double Pn, double tau, double q) {
  double lo = 0.0, hi = fmin(Pn / m, pow(Pn / tau, 1.0 / (q - 1.0)));
  double t = hi;
  for (int it = 0; it < 200; ++it) {
    const double tq2 = pow(t, q - 2.0);
    const double gt = m * t + tau * tq2 * t - Pn;
    if (gt < 0.0) lo = t; else hi = t;
    if (gt == 0.0 || hi - lo <= 4e-16 * hi) break;
    const double dg = m + tau * (q - 1.0) * tq2;
    double tn = t - gt / dg;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const double step = fabs(tn - t);
    t = tn;
    if (step <= 1e-16 * t) break;
  }
  return t;
}

template <int NW>
__device__ void prox_cell_q(double mbar, const double (&wbar)[NW], double tau, double qp, double a1, double tb,
                            double c, double& m, double (&w)[NW]) {
  const double q = qp / (qp - 1.0);
  double P[NW];
  double P2 = 0.0;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const bool neg = __double_as_longlong(wbar[k]) < 0;
    P[k] = ((k & 1) ? neg : !neg) ? wbar[k] : 0.0;
    P2 = fma(P[k], P[k], P2);
  }
  const double Pn = sqrt(P2);
  const double B = fma(-tau, c, mbar);
  if (isnan(B) || isnan(Pn)) {  // NaN in, NaN out (the CP step norm reports it)
    m = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = m;
    return;
  }
  const double lim = (tau / qp) * pow(Pn / tau, qp);
  if (-B - lim >= 0.0) {
    m = 0.0;
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = 0.0;
    return;
  }
  double lo = 0.0, hi = fmax(B, 0.0) + lim;
  double x = 0.5 * hi, t = 0.0;
  for (int it = 0; it < 200; ++it) {
    t = Pn > 0.0 ? velocity_q(x, Pn, tau, q) : 0.0;
    const double tq = pow(t, q);
    const double hx = fma(tb, x * x, a1 * x) - B - (tau / qp) * tq;
    if (hx < 0.0) lo = x; else hi = x;
    if (hx == 0.0 || hi - lo <= 4e-16 * hi) break;
    const double dh = fma(2.0 * tb, x, a1) + (Pn > 0.0 ? tau * (q - 1.0) * tq / (x + tau * (q - 1.0) * pow(t, q - 2.0)) : 0.0);
    double xn = x - hx / dh;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    const double step = fabs(xn - x);
    x = xn;
    if (step <= 1e-16 * x) break;
  }
  m = x;
  t = Pn > 0.0 ? velocity_q(x, Pn, tau, q) : 0.0;
  const double s = Pn > 0.0 ? x * t / Pn : 0.0;
#pragma unroll
  for (int k = 0; k < NW; ++k) w[k] = s * P[k];
}

// Per-step constants of the prox (tau is the CP primal step).
struct ProxK {
  double tau, half_tau, half_itau, tb;  // tau, tau/2, 1/(2 tau), tau f_b
  float tauf, tbf;
  df taud, tbd;                         // tau, tau f_b as double-float pairs
  bool tau_ok;                          // tau inside the FP32 fast-path range
};

__device__ __forceinline__ ProxK prox_consts(double tau, double half_itau, double f_b) {
  ProxK k;
  k.tau = tau;
  k.half_tau = 0.5 * tau;
  k.half_itau = half_itau;
  k.tb = tau * f_b;
  k.tauf = (float)tau;
  k.tbf = (float)k.tb;
  k.taud = df_from_double(tau);
  k.tbd = df_from_double(k.tb);
  k.tau_ok = tau > 1e-15 && tau < 1e15;
  return k;
}

// Root of h(m) = a1 m + tau b m^2 - B - hP/(m + tau)^2 with a1 = 1 + tau a,
// B = m_bar - tau c and hP = tau |P|^2 / 2 (the scalar equation above, with
// the FP64 constants combined before any rounding), then w = m/(m + tau) P.
// FP64 issues at 1/64 of the FP32 rate on GB300, so the root is found in FP32
// and polished in double-float arithmetic (df64.cuh, ~48 bits) by Newton
// steps on
//   g(m) = h(m) (m + tau)^2 = (a1 m + tau b m^2 - B) (m + tau)^2 - hP,
// which has the sign of h (the bracket stays valid) and needs no reciprocal;
// g' = (a1 + 2 tau b m)(m + tau)^2 + 2 (a1 m + tau b m^2 - B)(m + tau) > 0 near
// the root (there a1 m + tau b m^2 - B = hP/(m + tau)^2 >= 0) and is taken in
// FP32, so each step shrinks the error by ~1e-7 (plus the quadratic term):
// from an FP32 root two steps reach the double-float resolution.  The polish
// stops after a step below 1e-9 relative and keeps the bracket, bisecting if
// a step leaves it.  Inputs outside the FP32 range take an FP64 Newton.
template <int NW>
__device__ __forceinline__ void prox_cell(double mbar, const double (&wbar)[NW], const ProxK& K, double a1,
                                          float a1f, const df& a1d, double c, double& m, double (&w)[NW]) {
  // projection onto K by sign tests on the bit patterns (no FP64 min/max)
  double P[NW];
  double P2 = 0.0;
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const bool neg = __double_as_longlong(wbar[q]) < 0;
    P[q] = ((q & 1) ? neg : !neg) ? wbar[q] : 0.0;
    P2 = fma(P[q], P[q], P2);
  }
  const double B = fma(-K.tau, c, mbar);
  const double hp0 = P2 * K.half_itau;  // |P|^2 / (2 tau)
  if (B + hp0 <= 0.0) {                 // h(0) = -B - |P|^2/(2 tau) >= 0
    m = 0.0;
#pragma unroll
    for (int q = 0; q < NW; ++q) w[q] = 0.0;
    return;
  }
  const double hi0 = fmax(B, 0.0) + hp0;
  const double hP = K.half_tau * P2;
  const float hif = (float)hi0, Bf = (float)B, hPf = (float)hP;
  const bool fp32_ok = K.tau_ok && hif < 1e15f && hPf < 1e30f && fabsf(Bf) < 1e30f;
  if (!fp32_ok) {
    const double x = newton_h64(B, hP, K.tau, a1, K.tb, hi0);
    m = x;
    const double s = x / (x + K.tau);
#pragma unroll
    for (int q = 0; q < NW; ++q) w[q] = s * P[q];
    return;
  }
  const df Bd = df_from_double(B), hPd = df_from_double(hP);
  df lo{0.0f, 0.0f}, hi = df_from_double(hi0);
  df x{newton_h32(hif, Bf, hPf, K.tauf, a1f, K.tbf), 0.0f};
  for (int it = 0; it < 100; ++it) {
    const df t = df_add_same(x, K.taud);
    const df t2 = df_mul(t, t);
    const df u = df_add_same(df_mul(K.tbd, x), a1d);  // a1 + tau b x
    const df v = df_sub(df_mul(u, x), Bd);            // a1 x + tau b x^2 - B
    const df gx = df_sub(df_mul(v, t2), hPd);
    if (gx.hi < 0.0f) lo = x; else hi = x;
    if (gx.hi == 0.0f) break;
    const float dg = fmaf(fmaf(2.0f * K.tbf, x.hi, a1f), t2.hi, 2.0f * v.hi * t.hi);
    const float dx = __fdiv_rn(gx.hi, dg);
    const df xn = df_add_f(x, -dx);
    if (df_le(lo, xn) && df_le(xn, hi)) {
      x = xn;
      if (fabsf(dx) <= 1e-9f * x.hi) break;
    } else {
      const df mid = df_add_same(lo, hi);
      x = df{0.5f * mid.hi, 0.5f * mid.lo};
      if (df_sub(hi, lo).hi <= 1e-14f * hi.hi) break;
    }
  }
  // s = x / (x + tau): FP32 reciprocal refined once in double-float
  const df t = df_add_same(x, K.taud);
  const float r0 = __frcp_rn(t.hi);
  const df e = df_sub(df{1.0f, 0.0f}, df_mul(t, df{r0, 0.0f}));  // 1 - t r0, ~1e-7
  const df r = df_add_f(df{r0 * e.hi, 0.0f}, r0);                // r0 (1 + e)
  m = df_to_double(x);
  const double s = df_to_double(df_mul(x, r));
#pragma unroll
  for (int q = 0; q < NW; ++q) w[q] = s * P[q];
}

// y, ybar hold c planes; z one plane set.  Cell e pairs (m^{k+1}, w^k).
// The lift x = C^T z is formed from the four one-sided differences of z, which
// serve both the fluxes (x_w = D^T-type differences / dx) and
//   K z = ax ((z - zE) - (zW - z)) + ay ((z - zN) - (zS - z));
// on a Neumann axis the neighbour index of an end point is the point itself,
// so the difference across the end (a flux slot of Sec. 4.3 that does not
// exist) is zero and K takes its one-sided form.  VN (viscosity field): nu K z
// becomes K_nu z = kf_yp dyp - kf_ym dym (+ x terms), the face coefficients of
// Geom::kfx / kfy.
template <int ACTX, bool GENQ, bool VN>
__global__ void __launch_bounds__(kThreads) k_prox_cp(Geom g, Coef cf, const double* __restrict__ z,
                                                      double* __restrict__ y, double* __restrict__ ybar,
                                                      const double* __restrict__ V,
                                                      const double* __restrict__ W, double* partials,
                                                      DevScalars* sc, cudaGraphConditionalHandle h,
                                                      int use_handle, double* __restrict__ Az,
                                                      const double* __restrict__ rfin) {
  constexpr int NW = ACTX ? 4 : 2;
  const long long n = g.n;
  const double tau = sc->tau, theta = sc->theta;
  const ProxK K = prox_consts(tau, sc->half_itau, cf.f_b);
  const double t_nu = tau * g.nu, t_idt = tau * g.idt, t_idx = tau * g.idx, t_idy = tau * g.idy;
  const double a1_in = fma(tau, cf.f_a, 1.0), a1_last = fma(tau, fma(cf.g_a, g.idt, cf.f_a), 1.0);
  const float a1f_in = (float)a1_in, a1f_last = (float)a1_last;
  const df a1d_in = df_from_double(a1_in), a1d_last = df_from_double(a1_last);
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.ny);
    const long long t = e / g.ny;
    const int i = (int)(t % g.nx);
    const int k = (int)(t / g.nx);
    const long long base = (long long)k * g.S;
    const long long rowi = base + (long long)i * g.ny;
    const int jm = j == 0 ? (g.pery ? g.ny - 1 : 0) : j - 1;
    const int jp = j == g.ny - 1 ? (g.pery ? 0 : g.ny - 1) : j + 1;
    const double zc = z[e];
    if (Az != nullptr) Az[e] -= rfin[e];  // AAt z_{l+1} = b - r_final (stop reference)
    const double dyp = zc - z[rowi + jp], dym = z[rowi + jm] - zc;
    const long long f0 = (long long)i * g.ny;
    double Kz = VN ? fma(g.kfy[f0 + j], dyp, -g.kfy[f0 + jm] * dym) : g.ay * (dyp - dym);
    double d[NW];
    if (ACTX) {
      const int im = i == 0 ? (g.perx ? g.nx - 1 : 0) : i - 1;
      const int ip = i == g.nx - 1 ? (g.perx ? 0 : g.nx - 1) : i + 1;
      const double dxp = zc - z[base + (long long)ip * g.ny + j], dxm = z[base + (long long)im * g.ny + j] - zc;
      if (VN)
        Kz = fma(g.kfx[f0 + j], dxp, fma(-g.kfx[(long long)im * g.ny + j], dxm, Kz));
      else
        Kz = fma(g.ax, dxp - dxm, Kz);
      d[0] = dxp; d[1] = dxm; d[2] = dyp; d[3] = dym;
    } else {
      d[0] = dyp; d[1] = dym;
    }
    const double zn = (k + 1 < g.nt) ? z[e + g.S] : 0.0;
    // primal step y - tau x, x_m = nu K z + (z - z_next)/dt, x_w = d / dx
    const double m_old = y[e];
    const double mbar = fma(VN ? -tau : -t_nu, Kz, fma(-t_idt, zc - zn, m_old));
    double w_old[NW], wbar[NW], w_new[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      w_old[q] = y[e + (q + 1) * n];
      wbar[q] = fma(-((ACTX && q < 2) ? t_idx : t_idy), d[q], w_old[q]);
    }
    const bool last = (k == g.nt - 1);
    const long long f = (long long)i * g.ny + j;
    const double cc = last ? fma(W[f], g.idt, V[f]) : V[f];
    double m_new;
    if constexpr (GENQ)
      prox_cell_q<NW>(mbar, wbar, tau, cf.qprime, last ? a1_last : a1_in, K.tb, cc, m_new, w_new);
    else
      prox_cell<NW>(mbar, wbar, K, last ? a1_last : a1_in, last ? a1f_last : a1f_in, last ? a1d_last : a1d_in, cc,
                    m_new, w_new);
    const double dm = m_new - m_old;
    y[e] = m_new;
    ybar[e] = fma(theta, dm, m_new);
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      y[e + (q + 1) * n] = w_new[q];
      ybar[e + (q + 1) * n] = fma(theta, w_new[q] - w_old[q], w_new[q]);
    }
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
    const double tau_next = theta * tau;
    sc->tau = tau_next;
    sc->sigma = sc->sigma / theta;
    sc->theta = 1.0 / sqrt(1.0 + 2.0 * cf.gamma * tau_next);
    sc->half_itau = 0.5 / tau_next;
    sc->ell += 1;
    sc->cp_iters += 1;
    sc->cg_total += sc->cg_it;
    if (sc->cg_it > sc->cg_max) sc->cg_max = sc->cg_it;
    sc->cp_left -= 1;
    if (!isfinite(r)) {
      sc->status = MFG_ERR_NONFINITE;
      sc->cp_done = 1;
    }
    // a non-finite value or a timed-out device wait ends the instance's solve
    if (sc->status == MFG_ERR_NONFINITE || sc->status == MFG_ERR_TIMEOUT) sc->cp_done = 1;
    if (sc->cp_tol > 0.0 && r <= sc->cp_tol) sc->cp_done = 1;
    if (use_handle) cudaGraphSetConditional(h, (sc->cp_left > 0 && !sc->cp_done) ? 1u : 0u);
    sc->counter = 0;
  }
}

template <int ACTX, bool GENQ>
__global__ void __launch_bounds__(kThreads) k_prox_plain(Geom g, Coef cf, double tau,
                                                         const double* v, double* y,
                                                         const double* __restrict__ V,
                                                         const double* __restrict__ W) {
  constexpr int NW = ACTX ? 4 : 2;
  const long long n = g.n;
  const ProxK K = prox_consts(tau, 0.5 / tau, cf.f_b);
  const double a1_in = fma(tau, cf.f_a, 1.0), a1_last = fma(tau, fma(cf.g_a, g.idt, cf.f_a), 1.0);
  const float a1f_in = (float)a1_in, a1f_last = (float)a1_last;
  const df a1d_in = df_from_double(a1_in), a1d_last = df_from_double(a1_last);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / g.S);
    const long long f = e % g.S;
    double wbar[NW], w_new[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) wbar[q] = v[e + (q + 1) * n];
    const bool last = (k == g.nt - 1);
    const double cc = last ? fma(W[f], g.idt, V[f]) : V[f];
    double m_new;
    if constexpr (GENQ)
      prox_cell_q<NW>(v[e], wbar, tau, cf.qprime, last ? a1_last : a1_in, K.tb, cc, m_new, w_new);
    else
      prox_cell<NW>(v[e], wbar, K, last ? a1_last : a1_in, last ? a1f_last : a1f_in, last ? a1d_last : a1d_in, cc,
                    m_new, w_new);
    y[e] = m_new;
#pragma unroll
    for (int q = 0; q < NW; ++q) y[e + (q + 1) * n] = w_new[q];
  }
}

// One wave of resident blocks per instantiation (SMs x blocks per SM from the
// occupancy calculator), set by prox_configure: the prox step is FP64-bound
// with ~100 registers a thread, so a grid past one wave only adds a tail.
int g_prox_wave[8] = {kRedBlocks, kRedBlocks, kRedBlocks, kRedBlocks, kRedBlocks, kRedBlocks, kRedBlocks,
                      kRedBlocks};

int prox_configure() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MFG_ERR_CUDA;
  const void* fns[8] = {(const void*)k_prox_cp<0, false, false>, (const void*)k_prox_cp<0, false, true>,
                        (const void*)k_prox_cp<0, true, false>,  (const void*)k_prox_cp<0, true, true>,
                        (const void*)k_prox_cp<1, false, false>, (const void*)k_prox_cp<1, false, true>,
                        (const void*)k_prox_cp<1, true, false>,  (const void*)k_prox_cp<1, true, true>};
  for (int i = 0; i < 8; ++i) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[i], kThreads, 0) != cudaSuccess) return MFG_ERR_CUDA;
    g_prox_wave[i] = std::max(1, std::min(kVecBlocksMax, sms * std::max(occ, 1)));
  }
  return MFG_OK;
}

void launch_prox_cp(const Geom& g, const Coef& cf, const double* z, double* y, double* ybar,
                    const double* V, const double* W, double* partials, DevScalars* sc,
                    cudaGraphConditionalHandle h, int use_handle, cudaStream_t s, double* Az,
                    const double* rfin) {
  const int idx = (g.actx ? 4 : 0) + (cf.qprime != 2.0 ? 2 : 0) + (g.kfy != nullptr ? 1 : 0);
  const int nb = red_blocks(g.n, g_prox_wave[idx]);
  // the general-q' root finder and the viscosity field are their own
  // instantiations, so the q' = 2, constant-nu kernel keeps its registers
#define MFG_PROX_CP(A, Q, N) \
  k_prox_cp<A, Q, N><<<nb, kThreads, 0, s>>>(g, cf, z, y, ybar, V, W, partials, sc, h, use_handle, Az, rfin)
  const bool gq = cf.qprime != 2.0, vn = g.kfy != nullptr;
  if (g.actx) {
    if (gq) { if (vn) MFG_PROX_CP(1, true, true); else MFG_PROX_CP(1, true, false); }
    else    { if (vn) MFG_PROX_CP(1, false, true); else MFG_PROX_CP(1, false, false); }
  } else {
    if (gq) { if (vn) MFG_PROX_CP(0, true, true); else MFG_PROX_CP(0, true, false); }
    else    { if (vn) MFG_PROX_CP(0, false, true); else MFG_PROX_CP(0, false, false); }
  }
#undef MFG_PROX_CP
}

void launch_prox_plain(const Geom& g, const Coef& cf, double tau, const double* v, double* y,
                       const double* V, const double* W, cudaStream_t s) {
  const int nb = red_blocks(g.n, g.vec_blocks);
  if (cf.qprime != 2.0) {
    if (g.actx)
      k_prox_plain<1, true><<<nb, kThreads, 0, s>>>(g, cf, tau, v, y, V, W);
    else
      k_prox_plain<0, true><<<nb, kThreads, 0, s>>>(g, cf, tau, v, y, V, W);
  } else if (g.actx) {
    k_prox_plain<1, false><<<nb, kThreads, 0, s>>>(g, cf, tau, v, y, V, W);
  } else {
    k_prox_plain<0, false><<<nb, kThreads, 0, s>>>(g, cf, tau, v, y, V, W);
  }
}

}  // namespace mfg
