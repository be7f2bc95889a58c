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
#include <algorithm>

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
// mode 2: PCG step of the adjoint Schur system: r = C v, reduces pdot.r,
//         alpha = rz/(pdot.r).
// mode 3: adjoint right-hand side r = C v; reduces ||r||^2, resets the PCG
//         state with the fixed tolerance.
template <int ACTX>
__global__ void __launch_bounds__(kThreads) k_apply_C(Geom g, const double* __restrict__ v,
                                                      double* __restrict__ r, double alpha,
                                                      const double* __restrict__ m0,
                                                      const double* __restrict__ pdot,
                                                      double* partials, DevScalars* sc, int mode) {
  if (mode == 2 && sc->cg_done) return;
  if (mode == 1) alpha = sc->sigma;
  const long long n = g.n;
  const double* m = v;
  const double* wx1 = v + n;
  const double* wx2 = v + 2 * n;
  const double* wy1 = ACTX ? v + 3 * n : v + n;
  const double* wy2 = ACTX ? v + 4 * n : v + 2 * n;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.ny);
    const long long t = e / g.ny;
    const int i = (int)(t % g.nx);
    const int k = (int)(t / g.nx);
    const long long base = (long long)k * g.S;
    const Nb by = nbr(j, g.ny, g.pery);
    const long long rowi = base + (long long)i * g.ny;
    const double mc = m[e];
    double Km = g.ay * ((by.hm ? mc - m[rowi + by.im] : 0.0) + (by.hp ? mc - m[rowi + by.ip] : 0.0));
    double bw = g.idy * ((by.hp ? wy1[e] : 0.0) - (by.hm ? wy1[rowi + by.im] : 0.0) +
                         (by.hp ? wy2[rowi + by.ip] : 0.0) - (by.hm ? wy2[e] : 0.0));
    if (ACTX) {
      const Nb bx = nbr(i, g.nx, g.perx);
      const long long em = base + (long long)bx.im * g.ny + j, ep = base + (long long)bx.ip * g.ny + j;
      Km += g.ax * ((bx.hm ? mc - m[em] : 0.0) + (bx.hp ? mc - m[ep] : 0.0));
      bw += g.idx * ((bx.hp ? wx1[e] : 0.0) - (bx.hm ? wx1[em] : 0.0) + (bx.hp ? wx2[ep] : 0.0) -
                     (bx.hm ? wx2[e] : 0.0));
    }
    double val = g.nu * Km + mc * g.idt + bw;
    if (k >= 1) val -= m[e - g.S] * g.idt;
    if (m0 != nullptr && k == 0) val -= m0[(long long)i * g.ny + j] * g.idt;
    val *= alpha;
    r[e] = val;
    acc += (mode == 2) ? pdot[e] * val : val * val;
  }
  if (mode == 0) return;
  double part[1] = {acc};
  block_sum<1>(part);
  if (!publish_and_check_last<1>(part, partials, &sc->counter)) return;
  double tot[1];
  gather_partials<1>(partials, tot);
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
    sc->bnorm2 = tot[0];
    sc->cg_it = 0;
    // The paper's adaptive rule, min{1e-4, max{1e-6, 1e-4 r}} (Sec. 5).
    double tol = sc->cg_tol_fixed;
    if (sc->cg_rule == MFG_CG_ADAPTIVE) tol = fmin(1e-4, fmax(1e-6, 1e-4 * sc->r_last));
    sc->cg_tol = tol;
    sc->cg_done = !(tot[0] > 0.0);  // also true for NaN: flagged below
    if (!isfinite(tot[0])) {
      sc->cg_done = 1;
      sc->status = MFG_ERR_NONFINITE;
    }
    sc->counter = 0;
  }
}

void launch_apply_C(const Geom& g, const double* v, double* r, double alpha, const double* m0,
                    double* partials, DevScalars* sc, int mode, cudaStream_t s, const double* pdot) {
  const int nb = red_blocks(g.n);
  if (g.actx)
    k_apply_C<1><<<nb, kThreads, 0, s>>>(g, v, r, alpha, m0, pdot, partials, sc, mode);
  else
    k_apply_C<0><<<nb, kThreads, 0, s>>>(g, v, r, alpha, m0, pdot, partials, sc, mode);
}

// ----------------------------------------------------------------- C^T p --
// x_m^k = L p^k - p^{k+1}/dt (p^{N_t} := 0),  x_w^k = B^T p^k = -D_h p^k.
template <int ACTX>
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
    double Kp = g.ay * ((by.hm ? pc - pjm : 0.0) + (by.hp ? pc - pjp : 0.0));
    xy1[e] = by.hp ? (pc - pjp) * g.idy : 0.0;
    xy2[e] = by.hm ? (pjm - pc) * g.idy : 0.0;
    if (ACTX) {
      const Nb bx = nbr(i, g.nx, g.perx);
      const double pim = p[base + (long long)bx.im * g.ny + j], pip = p[base + (long long)bx.ip * g.ny + j];
      Kp += g.ax * ((bx.hm ? pc - pim : 0.0) + (bx.hp ? pc - pip : 0.0));
      xx1[e] = bx.hp ? (pc - pip) * g.idx : 0.0;
      xx2[e] = bx.hm ? (pim - pc) * g.idx : 0.0;
    }
    const double pn = (k + 1 < g.nt) ? p[e + g.S] : 0.0;
    xm[e] = g.nu * Kp + (pc - pn) * g.idt;
  }
}

void launch_apply_Ct(const Geom& g, const double* p, double* x, cudaStream_t s) {
  const int nb = red_blocks(g.n);
  if (g.actx)
    k_apply_Ct<1><<<nb, kThreads, 0, s>>>(g, p, x);
  else
    k_apply_Ct<0><<<nb, kThreads, 0, s>>>(g, p, x);
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
};

AatCoef aat_coef(const Geom& g) {
  const double ax = g.actx ? g.ax : 0.0, ay = g.ay, cK = 2.0 * (ax + ay);
  const double dt = 1.0 / g.idt, idt2 = g.idt * g.idt;
  return AatCoef{ax, ay, cK, g.nu * dt, g.nu * ay * g.idt, g.nu * ax * g.idt, g.nu * cK * g.idt + idt2, idt2};
}

int aat2_chunk(const Geom& g) {
  const long long cols = (long long)((g.ny + AJ - 1) / AJ) * ((g.nx + AI - 1) / AI);
  const long long want = 152 * 8;  // 256-thread blocks: 8 per SM fill it
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

template <int ACTX>
__global__ void __launch_bounds__(AJ * AI) k_aat_x(Geom g, AatCoef a, int kc, const double* __restrict__ p,
                                                   double* __restrict__ X, double* __restrict__ KP,
                                                   const DevScalars* sc, int mode) {
  if (mode == 1 && sc->cg_done) return;
  const int j = blockIdx.x * AJ + threadIdx.x, i = blockIdx.y * AI + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int k0 = blockIdx.z * kc, k1 = min(g.nt, k0 + kc);
  const Cols nb = aat_cols(g, i, j);
  const long long row = (long long)i * g.ny;
  long long base = (long long)k0 * g.S;
  double c = p[base + row + j];
  for (int k = k0; k < k1; ++k) {
    const double pn = (k + 1 < g.nt) ? p[base + g.S + row + j] : 0.0;
    double t = a.ay * (p[base + row + nb.jm] + p[base + row + nb.jp]);
    if (ACTX) t = fma(a.ax, p[base + (long long)nb.im * g.ny + j] + p[base + (long long)nb.ip * g.ny + j], t);
    const double kp = fma(a.cK, c, -t);
    X[base + row + j] = fma(a.ndt, kp, c - pn);
    KP[base + row + j] = kp;
    c = pn;
    base += g.S;
  }
}

// mode 0: q = AAt p.  mode 1 (PCG step): also reduces p.q and sets
// alpha = rz/(p.q) in the device scalars.
template <int ACTX>
__global__ void __launch_bounds__(AJ * AI) k_aat_q(Geom g, AatCoef a, int kc, const double* __restrict__ X,
                                                   const double* __restrict__ KP, const double* __restrict__ p,
                                                   double* __restrict__ q, double* partials, DevScalars* sc,
                                                   int mode) {
  if (mode == 1 && sc->cg_done) return;
  const int j = blockIdx.x * AJ + threadIdx.x, i = blockIdx.y * AI + threadIdx.y;
  double acc = 0.0;
  if (i < g.nx && j < g.ny) {
    const int k0 = blockIdx.z * kc, k1 = min(g.nt, k0 + kc);
    const Cols nb = aat_cols(g, i, j);
    const long long row = (long long)i * g.ny;
    long long base = (long long)k0 * g.S;
    double xprev = k0 > 0 ? X[base - g.S + row + j] : 0.0;
    for (int k = k0; k < k1; ++k) {
      const double xc = X[base + row + j];
      double t = a.c1 * (X[base + row + nb.jm] + X[base + row + nb.jp]);
      if (ACTX) t = fma(a.c2, X[base + (long long)nb.im * g.ny + j] + X[base + (long long)nb.ip * g.ny + j], t);
      t = fma(a.idt2, xprev, t);
      t = fma(-2.0, KP[base + row + j], t);
      const double qv = fma(a.c4, xc, -t);
      q[base + row + j] = qv;
      if (mode == 1) acc = fma(qv, p[base + row + j], acc);
      xprev = xc;
      base += g.S;
    }
  }
  if (mode != 1) return;
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

// Fused one-pass stencil on shared-memory tiles, used by the double-float
// variant: a block owns a TI x TJ spatial tile and marches over a chunk of
// planes; p planes are staged with a 2-point halo, xm with a 1-point halo (on
// a Neumann axis the halos hold mirror images; xm halo slots outside the
// domain are refreshed from their mirrors after xm is formed).
constexpr int TI = 16, TJ = 32;
constexpr int H2I = TI + 4, H2J = TJ + 4;  // p tile with halo 2
constexpr int H1I = TI + 2, H1J = TJ + 2;  // xm tile with halo 1

int aat_chunk(const Geom& g) {
  const long long tiles = (long long)((g.ny + TJ - 1) / TJ) * ((g.nx + TI - 1) / TI);
  long long want = 152 * 4;
  long long chunks = (want + tiles - 1) / tiles;
  if (chunks < 1) chunks = 1;
  if (chunks > g.nt) chunks = g.nt;
  int kc = (int)((g.nt + chunks - 1) / chunks);
  if (kc < 2) kc = 2;
  if (kc > g.nt) kc = g.nt;
  return kc;
}

int aat_blocks(const Geom& g) {
  const int kc = aat_chunk(g);
  const long long one = (long long)((g.ny + TJ - 1) / TJ) * ((g.nx + TI - 1) / TI) * ((g.nt + kc - 1) / kc);
  const dim3 g2 = aat2_grid(g, aat2_chunk(g));
  const long long two = (long long)g2.x * g2.y * g2.z;
  return (int)std::max(one, two);
}

// Index of grid point i on an axis: wrapped when periodic, mirrored across the
// end when Neumann (i = -1 -> 0, -2 -> 1, N -> N-1, N+1 -> N-2).
__device__ __forceinline__ int halo_index(int i, int N, int per) {
  if (i >= 0 && i < N) return i;
  if (per) {
    i %= N;
    return i < 0 ? i + N : i;
  }
  int m = i < 0 ? -1 - i : 2 * N - 1 - i;
  return m < 0 ? 0 : (m >= N ? N - 1 : m);
}

// The double-float version (df64.cuh): p is split into FP32 pairs as it is
// staged, every stencil operation runs on FP32 pairs, and q is rebuilt in FP64
// (one FP64 add per point) together with the FP64 p.q.
// About 48 significant bits; used by the MFG_MIXED_DF precision.
__device__ __forceinline__ void load_plane_h2_df(const Geom& g, const double* __restrict__ p, int k,
                                                 int i0, int j0, df (*dst)[H2J]) {
  const int tid = threadIdx.x + TJ * threadIdx.y;
  if (k >= g.nt) {
    for (int s = tid; s < H2I * H2J; s += TI * TJ) dst[s / H2J][s % H2J] = df{0.0f, 0.0f};
    return;
  }
  const double* pk = p + (long long)k * g.S;
  for (int s = tid; s < H2I * H2J; s += TI * TJ) {
    const int li = s / H2J, lj = s % H2J;
    const int gi = halo_index(i0 + li - 2, g.nx, g.perx);
    const int gj = halo_index(j0 + lj - 2, g.ny, g.pery);
    dst[li][lj] = df_from_double(pk[(long long)gi * g.ny + gj]);
  }
}

template <int ACTX, int WID>
__device__ __forceinline__ df fast_K_df(const df (*A)[WID], int r, int c, df ax, df ay, df cK) {
  df t = df_mul(ay, df_add(A[r][c - 1], A[r][c + 1]));
  if (ACTX) t = df_add(t, df_mul(ax, df_add(A[r - 1][c], A[r + 1][c])));
  return df_sub(df_mul(cK, A[r][c]), t);
}

template <int ACTX>
__global__ void __launch_bounds__(TI * TJ, 2) k_AAt_df(Geom g, int kc, const double* __restrict__ p,
                                                       double* __restrict__ q, double* partials,
                                                       DevScalars* sc, int mode) {
  if (mode == 1 && sc->cg_done) return;
  __shared__ df P[2][H2I][H2J];
  __shared__ df XM[H1I][H1J];
  __shared__ df KP[TI][TJ];
  const int tj = threadIdx.x, ti = threadIdx.y;
  const int j0 = blockIdx.x * TJ, i0 = blockIdx.y * TI;
  const int k0 = blockIdx.z * kc;
  const int k1 = min(g.nt, k0 + kc);
  const int gi = i0 + ti, gj = j0 + tj;
  const bool own = gi < g.nx && gj < g.ny;
  const double axd = ACTX ? g.ax : 0.0, ayd = g.ay, cKd = 2.0 * (axd + ayd);
  const df ax = df_from_double(axd), ay = df_from_double(ayd), cK = df_from_double(cKd);
  const df nax = df_from_double(g.nu * axd), nay = df_from_double(g.nu * ayd),
           ncK = df_from_double(g.nu * cKd);
  const df nu = df_from_double(g.nu), idt = df_from_double(g.idt), two = df{2.0f, 0.0f};
  const bool ghost_x = ACTX && !g.perx && (i0 == 0 || i0 + TI >= g.nx);
  const bool ghost_y = !g.pery && (j0 == 0 || j0 + TJ >= g.ny);
  const bool ghosts = ghost_x || ghost_y;
  const int tid = tj + TJ * ti;

  int cur = 0;
  load_plane_h2_df(g, p, k0, i0, j0, P[cur]);
  df xprev{0.0f, 0.0f};
  if (k0 > 0) {
    load_plane_h2_df(g, p, k0 - 1, i0, j0, P[cur ^ 1]);
    __syncthreads();
    if (own)
      xprev = df_add(fast_K_df<ACTX, H2J>(P[cur ^ 1], ti + 2, tj + 2, nax, nay, ncK),
                     df_mul(df_sub(P[cur ^ 1][ti + 2][tj + 2], P[cur][ti + 2][tj + 2]), idt));
    __syncthreads();
  }
  double acc = 0.0;
  for (int k = k0; k < k1; ++k) {
    load_plane_h2_df(g, p, k + 1, i0, j0, P[cur ^ 1]);
    __syncthreads();
    const df (*Pk)[H2J] = P[cur];
    const df (*Pn)[H2J] = P[cur ^ 1];
    for (int s = tid; s < H1I * H1J; s += TI * TJ) {
      const int li = s / H1J, lj = s % H1J;
      const df kp = fast_K_df<ACTX, H2J>(Pk, li + 1, lj + 1, ax, ay, cK);
      XM[li][lj] = df_add(df_mul(nu, kp), df_mul(df_sub(Pk[li + 1][lj + 1], Pn[li + 1][lj + 1]), idt));
      if (li >= 1 && li <= TI && lj >= 1 && lj <= TJ) KP[li - 1][lj - 1] = kp;
    }
    __syncthreads();
    if (ghosts) {
      for (int s = tid; s < H1I * H1J; s += TI * TJ) {
        const int li = s / H1J, lj = s % H1J;
        const int xi = i0 + li - 1, xj = j0 + lj - 1;
        const bool ox = ghost_x && (xi < 0 || xi >= g.nx);
        const bool oy = ghost_y && (xj < 0 || xj >= g.ny);
        if (ox || oy) {
          const int mi = ox ? (xi < 0 ? li + 1 : li - 1) : li;
          const int mj = oy ? (xj < 0 ? lj + 1 : lj - 1) : lj;
          XM[li][lj] = XM[mi][mj];
        }
      }
      __syncthreads();
    }
    if (own) {
      const df c = XM[ti + 1][tj + 1];
      const df nKxm = fast_K_df<ACTX, H1J>(XM, ti + 1, tj + 1, nax, nay, ncK);
      const df val = df_add(df_mul(two, KP[ti][tj]), df_add(df_mul(df_sub(c, xprev), idt), nKxm));
      xprev = c;
      const long long e = (long long)k * g.S + (long long)gi * g.ny + gj;
      const double vd = df_to_double(val);
      q[e] = vd;
      acc = fma(vd, p[e], acc);
    }
    __syncthreads();
    cur ^= 1;
  }
  if (mode != 1) return;
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
  if (df64) {
    const int kc = aat_chunk(g);
    dim3 grid((g.ny + TJ - 1) / TJ, (g.nx + TI - 1) / TI, (g.nt + kc - 1) / kc);
    dim3 block(TJ, TI);
    if (g.actx)
      k_AAt_df<1><<<grid, block, 0, s>>>(g, kc, p, q, partials, sc, mode);
    else
      k_AAt_df<0><<<grid, block, 0, s>>>(g, kc, p, q, partials, sc, mode);
    return;
  }
  const AatCoef a = aat_coef(g);
  const int kc = aat2_chunk(g);
  const dim3 grid = aat2_grid(g, kc), block(AJ, AI);
  double* X = scratch;
  double* KP = scratch + g.n;
  if (g.actx) {
    k_aat_x<1><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
    k_aat_q<1><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
  } else {
    k_aat_x<0><<<grid, block, 0, s>>>(g, a, kc, p, X, KP, sc, mode);
    k_aat_q<0><<<grid, block, 0, s>>>(g, a, kc, X, KP, p, q, partials, sc, mode);
  }
}

int aat_kernel_count(int df64) { return df64 ? 1 : 2; }

}  // namespace mfg
