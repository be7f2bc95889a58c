// Space-time stencils of the discrete Fokker-Planck constraint:
//   C v      (eq. ABC, reduced), the CP right-hand side sigma (C ybar - d),
//   C^T p    (its transpose),
//   C C^T p  (eq. largeA), in two halo-free passes over p.
//
// Row k of C (plane k, time level k+1) reads
//   L m^{k+1} - m^k/dt + div_h w^k,  L = nu K + I/dt   (Sec. 3, matrices A, B)
// with K the negative 5-point Laplacian and div_h the divergence of Sec. 2,
// D^1/D^2 blocks of Sec. 4.3 per axis.  On a Neumann axis the blocks have no
// entries past the ends; on a periodic axis indices wrap.  Both cases use one
// rule: a point has a "minus" neighbour (hm) and a "plus" neighbour (hp) unless
// it sits at the matching end of a Neumann axis.
#include "df64.cuh"
#include "mfg_internal.cuh"
#include "reduce.cuh"

namespace mfg {

struct Nb {
  int im, ip;
  bool hm, hp;
};

__device__ __forceinline__ Nb nbr(int i, int N, int per) {
  Nb b;
  if (per) {
    b.im = (i == 0) ? N - 1 : i - 1;
    b.ip = (i == N - 1) ? 0 : i + 1;
    b.hm = b.hp = true;
  } else {
    b.hm = i >= 1;
    b.hp = i <= N - 2;
    b.im = b.hm ? i - 1 : i;
    b.ip = b.hp ? i + 1 : i;
  }
  return b;
}

__device__ __forceinline__ int wrap_or_neg(int i, int N, int per) {
  if (i >= 0 && i < N) return i;
  if (!per) return -1;
  i %= N;
  return i < 0 ? i + N : i;
}

// ------------------------------------------------------------------- C v --
// mode 0: r = alpha * (C v - d), d = m0/dt on plane 0 when m0 != nullptr.
// mode 1: CP right-hand side r = sigma (C v - d) with sigma from the device
//         scalars; reduces ||r||^2, resets the PCG state for the new solve.
//         With Az != nullptr (the MFG_CG_REF_RHS stop reference) Az holds
//         AAt z_l on entry and b = AAt z_l + r, the right-hand side of the
//         system of eq. CC*, on exit; ||b||^2 becomes the reference of the
//         relative tolerance, and a warm start already inside it stops the
//         solve before its first iteration.
// mode 2: PCG step of the adjoint Schur system: r = C v, reduces pdot.r,
//         alpha = rz/(pdot.r).
// mode 3: adjoint right-hand side r = C v; reduces ||r||^2, resets the PCG
//         state with the fixed tolerance.
// VN (viscosity field): nu K m becomes K_nu m = sum over the node's faces of
// kf (m - m_nb), kf the face coefficient of Geom::kfx / kfy; at a Neumann end
// the neighbour index is the node itself, so the missing face adds nothing.
template <int ACTX, bool VN>
__global__ void __launch_bounds__(kThreads) k_apply_C(Geom g, const double* __restrict__ v,
                                                      double* __restrict__ r, double alpha,
                                                      const double* __restrict__ m0,
                                                      const double* __restrict__ pdot,
                                                      double* partials, DevScalars* sc, int mode,
                                                      double* __restrict__ Az) {
  if (mode == 2 && sc->cg_done) return;
  if (mode == 1) alpha = sc->sigma;
  const long long n = g.n;
  const double* m = v;
  const double* wx1 = v + n;
  const double* wx2 = v + 2 * n;
  const double* wy1 = ACTX ? v + 3 * n : v + n;
  const double* wy2 = ACTX ? v + 4 * n : v + 2 * n;
  // alpha folded into the coefficients: r = alpha nu K m + alpha div_h w + alpha (m^k - m^{k-1})/dt
  const double anu = alpha * g.nu, ax = ACTX ? g.ax : 0.0;
  const double kc = anu * 2.0 * (ax + g.ay), kx = anu * ax, ky = anu * g.ay;
  const double aix = alpha * g.idx, aiy = alpha * g.idy, aidt = alpha * g.idt;
  double acc = 0.0, accb = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.ny);
    const long long t = e / g.ny;
    const int i = (int)(t % g.nx);
    const int k = (int)(t / g.nx);
    const long long base = (long long)k * g.S;
    const long long rowi = base + (long long)i * g.ny;
    // K m with the point itself as the missing neighbour at a Neumann end (one-sided rows)
    const Nb by = nbr(j, g.ny, g.pery);
    const double mc = m[e];
    double t1 = ky * (m[rowi + by.im] + m[rowi + by.ip]);
    // div_h w: flux slots past a Neumann end do not exist and read as zero
    const double sy = ((by.hp ? wy1[e] : 0.0) - (by.hm ? wy1[rowi + by.im] : 0.0)) +
                      ((by.hp ? wy2[rowi + by.ip] : 0.0) - (by.hm ? wy2[e] : 0.0));
    double val;
    double kvm = 0.0;  // K_nu m (VN)
    if (VN) {
      const long long f = (long long)i * g.ny;
      kvm = fma(g.kfy[f + j], mc - m[rowi + by.ip], g.kfy[f + by.im] * (mc - m[rowi + by.im]));
    }
    if (ACTX) {
      const Nb bx = nbr(i, g.nx, g.perx);
      const long long em = base + (long long)bx.im * g.ny + j, ep = base + (long long)bx.ip * g.ny + j;
      t1 = fma(kx, m[em] + m[ep], t1);
      const double sx = ((bx.hp ? wx1[e] : 0.0) - (bx.hm ? wx1[em] : 0.0)) +
                        ((bx.hp ? wx2[ep] : 0.0) - (bx.hm ? wx2[e] : 0.0));
      if (VN) {
        kvm = fma(g.kfx[(long long)i * g.ny + j], mc - m[ep], kvm);
        kvm = fma(g.kfx[(long long)bx.im * g.ny + j], mc - m[em], kvm);
        val = fma(aix, sx, fma(aiy, sy, alpha * kvm));
      } else {
        val = fma(aix, sx, fma(aiy, sy, fma(kc, mc, -t1)));
      }
    } else {
      val = VN ? fma(aiy, sy, alpha * kvm) : fma(aiy, sy, fma(kc, mc, -t1));
    }
    const double mprev = k >= 1 ? m[e - g.S] : (m0 != nullptr ? m0[(long long)i * g.ny + j] : 0.0);
    val = fma(aidt, mc - mprev, val);
    r[e] = val;
    acc = (mode == 2) ? fma(pdot[e], val, acc) : fma(val, val, acc);
    if (Az != nullptr) {
      const double b = Az[e] + val;
      Az[e] = b;
      accb = fma(b, b, accb);
    }
  }
  if (mode == 0) return;
  double part[2] = {acc, accb};
  block_sum<2>(part);
  if (!publish_and_check_last<2>(part, partials, &sc->counter)) return;
  double tot[2];
  gather_partials<2>(partials, tot);
  if (mode == 2) {
    if (flat_tid() == 0) {
      sc->pq = tot[0];
      if (tot[0] > 0.0 && isfinite(tot[0])) {
        sc->alpha = sc->rz / tot[0];
      } else {
        sc->alpha = 0.0;
        sc->cg_done = 1;
        if (sc->status == MFG_OK) sc->status = MFG_ERR_NONFINITE;
      }
      sc->counter = 0;
    }
    return;
  }
  if (flat_tid() == 0) {
    const double rr0 = tot[0], b2 = (Az != nullptr) ? tot[1] : tot[0];
    sc->bnorm2 = b2;  // reference of the relative tolerance: ||b||^2 or ||r_0||^2
    sc->rr = rr0;
    sc->cg_it = 0;
    // The paper's adaptive rule, min{1e-4, max{1e-6, 1e-4 r}} (Sec. 5).
    double tol = sc->cg_tol_fixed;
    if (sc->cg_rule == MFG_CG_ADAPTIVE) tol = fmin(1e-4, fmax(1e-6, 1e-4 * sc->r_last));
    sc->cg_tol = tol;
    // no iteration when r_0 = 0 or r_0 is already inside the tolerance (NaN: flagged below)
    sc->cg_done = !(rr0 > 0.0) || rr0 <= tol * tol * b2;
    if (!isfinite(rr0) || !isfinite(b2)) {
      sc->cg_done = 1;
      sc->status = MFG_ERR_NONFINITE;
    }
    sc->counter = 0;
  }
}

void launch_apply_C(const Geom& g, const double* v, double* r, double alpha, const double* m0,
                    double* partials, DevScalars* sc, int mode, cudaStream_t s, const double* pdot,
                    double* Az) {
  const int nb = red_blocks(g.n, g.vec_blocks);
  const bool vn = g.kfy != nullptr;
  if (g.actx && vn)
    k_apply_C<1, true><<<nb, kThreads, 0, s>>>(g, v, r, alpha, m0, pdot, partials, sc, mode, Az);
  else if (g.actx)
    k_apply_C<1, false><<<nb, kThreads, 0, s>>>(g, v, r, alpha, m0, pdot, partials, sc, mode, Az);
  else if (vn)
    k_apply_C<0, true><<<nb, kThreads, 0, s>>>(g, v, r, alpha, m0, pdot, partials, sc, mode, Az);
  else
    k_apply_C<0, false><<<nb, kThreads, 0, s>>>(g, v, r, alpha, m0, pdot, partials, sc, mode, Az);
}

// ----------------------------------------------------------------- C^T p --
// x_m^k = L p^k - p^{k+1}/dt (p^{N_t} := 0),  x_w^k = B^T p^k = -D_h p^k.
// VN: L = K_nu + I/dt with the face coefficients of Geom::kfx / kfy.
template <int ACTX, bool VN>
__global__ void __launch_bounds__(kThreads) k_apply_Ct(Geom g, const double* __restrict__ p,
                                                       double* __restrict__ x) {
  const long long n = g.n;
  double* xm = x;
  double* xx1 = x + n;
  double* xx2 = x + 2 * n;
  double* xy1 = ACTX ? x + 3 * n : x + n;
  double* xy2 = ACTX ? x + 4 * n : x + 2 * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.ny);
    const long long t = e / g.ny;
    const int i = (int)(t % g.nx);
    const int k = (int)(t / g.nx);
    const long long base = (long long)k * g.S;
    const long long rowi = base + (long long)i * g.ny;
    const Nb by = nbr(j, g.ny, g.pery);
    const double pc = p[e];
    const double pjm = p[rowi + by.im], pjp = p[rowi + by.ip];
    const long long f = (long long)i * g.ny;
    double Kp = VN ? fma(g.kfy[f + j], pc - pjp, g.kfy[f + by.im] * (pc - pjm))
                   : g.ay * ((by.hm ? pc - pjm : 0.0) + (by.hp ? pc - pjp : 0.0));
    xy1[e] = by.hp ? (pc - pjp) * g.idy : 0.0;
    xy2[e] = by.hm ? (pjm - pc) * g.idy : 0.0;
    if (ACTX) {
      const Nb bx = nbr(i, g.nx, g.perx);
      const double pim = p[base + (long long)bx.im * g.ny + j], pip = p[base + (long long)bx.ip * g.ny + j];
      if (VN)
        Kp = fma(g.kfx[f + j], pc - pip, fma(g.kfx[(long long)bx.im * g.ny + j], pc - pim, Kp));
      else
        Kp += g.ax * ((bx.hm ? pc - pim : 0.0) + (bx.hp ? pc - pip : 0.0));
      xx1[e] = bx.hp ? (pc - pip) * g.idx : 0.0;
      xx2[e] = bx.hm ? (pim - pc) * g.idx : 0.0;
    }
    const double pn = (k + 1 < g.nt) ? p[e + g.S] : 0.0;
    xm[e] = (VN ? Kp : g.nu * Kp) + (pc - pn) * g.idt;
  }
}

void launch_apply_Ct(const Geom& g, const double* p, double* x, cudaStream_t s) {
  const int nb = red_blocks(g.n, g.vec_blocks);
  const bool vn = g.kfy != nullptr;
  if (g.actx && vn)
    k_apply_Ct<1, true><<<nb, kThreads, 0, s>>>(g, p, x);
  else if (g.actx)
    k_apply_Ct<1, false><<<nb, kThreads, 0, s>>>(g, p, x);
  else if (vn)
    k_apply_Ct<0, true><<<nb, kThreads, 0, s>>>(g, p, x);
  else
    k_apply_Ct<0, false><<<nb, kThreads, 0, s>>>(g, p, x);
}

// ---------------------------------------------------------------- C C^T p --
// Factored form q = C (C^T p).  With xm^k = L p^k - p^{k+1}/dt (the m rows of
// C^T p) and B B^T = 2K (eq. precstead):
//   q^k = L xm^k - xm^{k-1}/dt + 2 K p^k        (xm^{-1} := 0).
//
// FP64 issue is the limit on GB300 (a warp's FP64 instruction takes 16 SM
// clocks; memory traffic is far below the HBM bound), so the stencil is laid
// out for the fewest FP64 instructions per point:
//   K u = cK u - ax (uW + uE) - ay (uN + uS),   cK = 2 (ax + ay)   (5 ops),
// and it runs in two halo-free passes over the grid, each point computed once:
//   pass 1:  kp = K p,   X = dt xm = fma(nu dt, kp, p^k - p^{k+1})        (7 ops)
//   pass 2:  q = c4 X - c2 (XW + XE) - c1 (XN + XS) - X^{k-1}/dt^2 + 2 kp (7 ops)
// with c1 = nu ay/dt, c2 = nu ax/dt, c4 = nu cK/dt + 1/dt^2, plus one FMA for
// p.q.  (A one-pass version that forms xm on a shared-memory tile must
// recompute it on the tile's halo and needs ~20 FP64 ops per point.)
// On a Neumann axis the neighbour index of an end point is the point itself
// (u_{-1} = u_0, u_N = u_{N-1}), which turns the same formula into the
// one-sided D^1 (D^1)^T rows of Sec. 4.3, for p and for X alike.
// Threads own one (i, j) column and march over a chunk of time planes, so
// p^{k+1} and X^{k-1} stay in registers from one plane to the next.
constexpr int AJ = 32, AI = 8;  // block = AJ x AI columns

struct AatCoef {
  double ax, ay, cK, ndt;      // pass 1
  double c1, c2, c4, idt2;     // pass 2
  double dt, idt;              // viscosity field (VN)
};

AatCoef aat_coef(const Geom& g) {
  const double ax = g.actx ? g.ax : 0.0, ay = g.ay, cK = 2.0 * (ax + ay);
  const double dt = 1.0 / g.idt, idt2 = g.idt * g.idt;
  return AatCoef{ax, ay, cK, g.nu * dt, g.nu * ay * g.idt, g.nu * ax * g.idt, g.nu * cK * g.idt + idt2, idt2,
                 dt, g.idt};
}



int aat2_chunk(const Geom& g) {
  const long long cols = (long long)((g.ny + AJ - 1) / AJ) * ((g.nx + AI - 1) / AI);
  const long long want = g.aat_want;  // default 152 * 8: 256-thread blocks, 8 per SM fill it
  long long chunks = (want + cols - 1) / cols;
  if (chunks < 1) chunks = 1;
  if (chunks > g.nt) chunks = g.nt;
  return (int)((g.nt + chunks - 1) / chunks);
}

dim3 aat2_grid(const Geom& g, int kc) {
  return dim3((g.ny + AJ - 1) / AJ, (g.nx + AI - 1) / AI, (g.nt + kc - 1) / kc);
}

struct Cols {
  int jm, jp, im, ip;
};

// Neighbour columns: wrapped on a periodic axis, the point itself at the end
// of a Neumann axis (and on an axis of length 1).
__device__ __forceinline__ Cols aat_cols(const Geom& g, int i, int j) {
  Cols c;
  c.jm = j == 0 ? (g.pery ? g.ny - 1 : 0) : j - 1;
  c.jp = j == g.ny - 1 ? (g.pery ? 0 : g.ny - 1) : j + 1;
  c.im = i == 0 ? (g.perx ? g.nx - 1 : 0) : i - 1;
  c.ip = i == g.nx - 1 ? (g.perx ? 0 : g.nx - 1) : i + 1;
  return c;
}

// Viscosity field (VN): with L = K_nu + I/dt the two passes read
//   pass 1:  kp = K p,  X = dt K_nu p + p^k - p^{k+1}
//   pass 2:  q = (K_nu X)/dt + (X - X^{k-1})/dt^2 + 2 kp,
// K_nu u = sum over the node's faces of kf (u - u_nb); the four face
// coefficients of a column are loaded once, before its march over the planes.
struct FaceCoef {
  double yp, ym, xp, xm;
};

__device__ __forceinline__ FaceCoef face_coef(const Geom& g, int i, int j, const Cols& nb, double scale) {
  FaceCoef f;
  const long long row = (long long)i * g.ny;
  f.yp = g.kfy[row + j] * scale;
  f.ym = g.kfy[row + nb.jm] * scale;
  f.xp = g.actx ? g.kfx[row + j] * scale : 0.0;
  f.xm = g.actx ? g.kfx[(long long)nb.im * g.ny + j] * scale : 0.0;
  return f;
}

template <int ACTX, bool VN>
__global__ void __launch_bounds__(AJ * AI) k_aat_x(Geom g, AatCoef a, int kc, const double* __restrict__ p,
                                                   double* __restrict__ X, double* __restrict__ KP,
                                                   const DevScalars* sc, int mode) {
  if (mode != 0 && sc->cg_done) return;
  const int j = blockIdx.x * AJ + threadIdx.x, i = blockIdx.y * AI + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int k0 = blockIdx.z * kc, k1 = min(g.nt, k0 + kc);
  const Cols nb = aat_cols(g, i, j);
  const long long row = (long long)i * g.ny;
  FaceCoef fc{0.0, 0.0, 0.0, 0.0};
  if (VN) fc = face_coef(g, i, j, nb, a.dt);
  long long base = (long long)k0 * g.S;
  double c = p[base + row + j];
  for (int k = k0; k < k1; ++k) {
    const double pn = (k + 1 < g.nt) ? p[base + g.S + row + j] : 0.0;
    const double pS = p[base + row + nb.jm], pN = p[base + row + nb.jp];
    double t = a.ay * (pS + pN);
    double pW = 0.0, pE = 0.0;
    if (ACTX) {
      pW = p[base + (long long)nb.im * g.ny + j];
      pE = p[base + (long long)nb.ip * g.ny + j];
      t = fma(a.ax, pW + pE, t);
    }
    const double kp = fma(a.cK, c, -t);
    if (VN) {
      double kv = fma(fc.yp, c - pN, fc.ym * (c - pS));  // dt K_nu p
      if (ACTX) kv = fma(fc.xp, c - pE, fma(fc.xm, c - pW, kv));
      X[base + row + j] = kv + (c - pn);
    } else {
      X[base + row + j] = fma(a.ndt, kp, c - pn);
    }
    KP[base + row + j] = kp;
    c = pn;
    base += g.S;
  }
}

// mode 0: q = AAt p.  mode 1 (PCG step): also reduces p.q and sets
// alpha = rz/(p.q) in the device scalars.
template <int ACTX, bool VN>
// 2-D: capped at 64 registers (four 256-thread blocks per SM) to hide the load latency
__global__ void __launch_bounds__(AJ * AI, (ACTX && !VN) ? 4 : 3) k_aat_q(Geom g, AatCoef a, int kc, const double* __restrict__ X,
                                                   const double* __restrict__ KP, const double* __restrict__ p,
                                                   double* __restrict__ q, double* partials, DevScalars* sc,
                                                   int mode) {
  if (mode != 0 && sc->cg_done) return;
  const int j = blockIdx.x * AJ + threadIdx.x, i = blockIdx.y * AI + threadIdx.y;
  double acc = 0.0;
  if (i < g.nx && j < g.ny) {
    const int k0 = blockIdx.z * kc, k1 = min(g.nt, k0 + kc);
    const Cols nb = aat_cols(g, i, j);
    const long long row = (long long)i * g.ny;
    FaceCoef fc{0.0, 0.0, 0.0, 0.0};
    if (VN) fc = face_coef(g, i, j, nb, a.idt);
    long long base = (long long)k0 * g.S;
    double xprev = k0 > 0 ? X[base - g.S + row + j] : 0.0;
    for (int k = k0; k < k1; ++k) {
      const double xc = X[base + row + j];
      double qv;
      if (VN) {
        const double xS = X[base + row + nb.jm], xN = X[base + row + nb.jp];
        double kv = fma(fc.yp, xc - xN, fc.ym * (xc - xS));  // K_nu X / dt
        if (ACTX) {
          const double xW = X[base + (long long)nb.im * g.ny + j], xE = X[base + (long long)nb.ip * g.ny + j];
          kv = fma(fc.xp, xc - xE, fma(fc.xm, xc - xW, kv));
        }
        qv = fma(2.0, KP[base + row + j], fma(a.idt2, xc - xprev, kv));
      } else {
        double t = a.c1 * (X[base + row + nb.jm] + X[base + row + nb.jp]);
        if (ACTX) t = fma(a.c2, X[base + (long long)nb.im * g.ny + j] + X[base + (long long)nb.ip * g.ny + j], t);
        t = fma(a.idt2, xprev, t);
        t = fma(-2.0, KP[base + row + j], t);
        qv = fma(a.c4, xc, -t);
      }
      q[base + row + j] = qv;
      if (mode == 1) acc = fma(qv, p[base + row + j], acc);
      xprev = xc;
      base += g.S;
    }
  }
  if (mode == 0) return;
  double part[1] = {acc};
  block_sum<1>(part);
  if (!publish_and_check_last<1>(part, partials, &sc->counter)) return;
  double tot[1];
  gather_partials<1>(partials, tot);
  if (flat_tid() == 0) {
    sc->pq = tot[0];
    if (tot[0] > 0.0 && isfinite(tot[0])) {
      sc->alpha = sc->rz / tot[0];
    } else {
      sc->alpha = 0.0;
      sc->cg_done = 1;
      if (sc->status == MFG_OK) sc->status = MFG_ERR_NONFINITE;
    }
    sc->counter = 0;
  }
}

int aat_blocks(const Geom& g) {
  const dim3 g2 = aat2_grid(g, aat2_chunk(g));
  return (int)((long long)g2.x * g2.y * g2.z);
}

// The same two passes in double-float arithmetic (df64.cuh, the MFG_MIXED_DF
// precision): p is split into FP32 pairs as it is loaded, every stencil
// operation runs on FP32 pairs, X and Kp are stored as pairs (8 bytes, like a
// double), and q is joined back to FP64 (one FP64 add) together with the FP64
// p.q.  About 48 significant bits; ~2 FP64 instructions per point instead of
// 15, the rest on the FP32 pipes.
__device__ __forceinline__ df df_scale2(df a) { return df{2.0f * a.hi, 2.0f * a.lo}; }

template <int ACTX>
__global__ void __launch_bounds__(AJ * AI) k_aat_x_df(Geom g, AatCoef ad, int kc, const double* __restrict__ p,
                                                      df* __restrict__ X, df* __restrict__ KP,
                                                      const DevScalars* sc, int mode) {
  if (mode != 0 && sc->cg_done) return;
  const int j = blockIdx.x * AJ + threadIdx.x, i = blockIdx.y * AI + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const df ax = df_from_double(ad.ax), ay = df_from_double(ad.ay), cK = df_from_double(ad.cK),
           ndt = df_from_double(ad.ndt);
  const int k0 = blockIdx.z * kc, k1 = min(g.nt, k0 + kc);
  const Cols nb = aat_cols(g, i, j);
  const long long row = (long long)i * g.ny;
  long long base = (long long)k0 * g.S;
  df c = df_from_double(p[base + row + j]);
  for (int k = k0; k < k1; ++k) {
    const df pn = (k + 1 < g.nt) ? df_from_double(p[base + g.S + row + j]) : df{0.0f, 0.0f};
    df t = df_mul(ay, df_add(df_from_double(p[base + row + nb.jm]), df_from_double(p[base + row + nb.jp])));
    if (ACTX)
      t = df_add(t, df_mul(ax, df_add(df_from_double(p[base + (long long)nb.im * g.ny + j]),
                                      df_from_double(p[base + (long long)nb.ip * g.ny + j]))));
    const df kp = df_sub(df_mul(cK, c), t);
    X[base + row + j] = df_add(df_mul(ndt, kp), df_sub(c, pn));
    KP[base + row + j] = kp;
    c = pn;
    base += g.S;
  }
}

template <int ACTX>
__global__ void __launch_bounds__(AJ * AI) k_aat_q_df(Geom g, AatCoef ad, int kc, const df* __restrict__ X,
                                                      const df* __restrict__ KP, const double* __restrict__ p,
                                                      double* __restrict__ q, double* partials, DevScalars* sc,
                                                      int mode) {
  if (mode != 0 && sc->cg_done) return;
  const int j = blockIdx.x * AJ + threadIdx.x, i = blockIdx.y * AI + threadIdx.y;
  double acc = 0.0;
  if (i < g.nx && j < g.ny) {
    const df c1 = df_from_double(ad.c1), c2 = df_from_double(ad.c2), c4 = df_from_double(ad.c4),
             idt2 = df_from_double(ad.idt2);
    const int k0 = blockIdx.z * kc, k1 = min(g.nt, k0 + kc);
    const Cols nb = aat_cols(g, i, j);
    const long long row = (long long)i * g.ny;
    long long base = (long long)k0 * g.S;
    df xprev = k0 > 0 ? X[base - g.S + row + j] : df{0.0f, 0.0f};
    for (int k = k0; k < k1; ++k) {
      const df xc = X[base + row + j];
      df t = df_mul(c1, df_add(X[base + row + nb.jm], X[base + row + nb.jp]));
      if (ACTX)
        t = df_add(t, df_mul(c2, df_add(X[base + (long long)nb.im * g.ny + j], X[base + (long long)nb.ip * g.ny + j])));
      t = df_add(t, df_mul(idt2, xprev));
      t = df_sub(t, df_scale2(KP[base + row + j]));
      const double qv = df_to_double(df_sub(df_mul(c4, xc), t));
      q[base + row + j] = qv;
      if (mode == 1) acc = fma(qv, p[base + row + j], acc);
      xprev = xc;
      base += g.S;
    }
  }
  if (mode == 0) return;
  double part[1] = {acc};
  block_sum<1>(part);
  if (!publish_and_check_last<1>(part, partials, &sc->counter)) return;
  double tot[1];
  gather_partials<1>(partials, tot);
  if (flat_tid() == 0) {
    sc->pq = tot[0];
    if (tot[0] > 0.0 && isfinite(tot[0])) {
      sc->alpha = sc->rz / tot[0];
    } else {
      sc->alpha = 0.0;
      sc->cg_done = 1;
      if (sc->status == MFG_OK) sc->status = MFG_ERR_NONFINITE;
    }
    sc->counter = 0;
  }
}

void launch_AAt(const Geom& g, const double* p, double* q, double* scratch, double* partials,
                DevScalars* sc, int mode, cudaStream_t s, int df64) {
  const AatCoef a = aat_coef(g);
  const int kc = aat2_chunk(g);
  const dim3 grid = aat2_grid(g, kc), block(AJ, AI);
  if (df64 && g.kfy == nullptr) {  // a viscosity field takes the FP64 stencil
    df* X = reinterpret_cast<df*>(scratch);
    df* KP = X + g.n;
    if (g.actx) {
      k_aat_x_df<1><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
      k_aat_q_df<1><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
    } else {
      k_aat_x_df<0><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
      k_aat_q_df<0><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
    }
    return;
  }
  double* X = scratch;
  double* KP = scratch + g.n;
  const bool vn = g.kfy != nullptr;
  if (g.actx && vn) {
    k_aat_x<1, true><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
    k_aat_q<1, true><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
  } else if (g.actx) {
    k_aat_x<1, false><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
    k_aat_q<1, false><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
  } else if (vn) {
    k_aat_x<0, true><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
    k_aat_q<0, true><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
  } else {
    k_aat_x<0, false><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
    k_aat_q<0, false><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
  }
}

int aat_kernel_count(int) { return 2; }

}  // namespace mfg
