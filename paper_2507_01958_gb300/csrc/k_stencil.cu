// Space-time stencils of the discrete Fokker-Planck constraint:
//   C v      (eq. ABC, reduced), the CP right-hand side sigma (C ybar - d),
//   C^T p    (its transpose),
//   C C^T p  (eq. largeA), fused in one pass over p.
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
// Fused factored form q = C (C^T p), marching in time over a chunk of planes.
// With xm^k = L p^k - p^{k+1}/dt and B B^T = 2K (eq. precstead):
//   q^k = L xm^k - xm^{k-1}/dt + 2 K p^k        (xm^{-1} := 0).
// A block owns a TI x TJ spatial tile; p planes are staged in shared memory
// with a 2-point halo, xm with a 1-point halo.  Each p plane is read from
// global memory once per tile (plus halo) instead of once per stencil point.
//
// FP64 issue is the limit on GB300 (1/58 of the FP32 rate), so the stencil is
// branch-free with the fewest FP64 instructions:
//   K u = cK u - ax (uW + uE) - ay (uN + uS),   cK = 2 (ax + ay),
// (5 FP64 ops; nu folded into the coefficients where only nu K u is needed).
// On a Neumann axis the halos hold mirror images (u_{-1} = u_0, u_N = u_{N-1}),
// which turns the same formula into the one-sided D^1 (D^1)^T rows of Sec. 4.3;
// xm halo slots outside the domain are refreshed from their mirrors after xm is
// formed.
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
  return ((g.ny + TJ - 1) / TJ) * ((g.nx + TI - 1) / TI) * ((g.nt + kc - 1) / kc);
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

__device__ __forceinline__ void load_plane_h2(const Geom& g, const double* __restrict__ p, int k,
                                              int i0, int j0, double (*dst)[H2J]) {
  const int tid = threadIdx.x + TJ * threadIdx.y;
  if (k >= g.nt) {
    for (int s = tid; s < H2I * H2J; s += TI * TJ) dst[s / H2J][s % H2J] = 0.0;
    return;
  }
  const double* pk = p + (long long)k * g.S;
  for (int s = tid; s < H2I * H2J; s += TI * TJ) {
    const int li = s / H2J, lj = s % H2J;
    const int gi = halo_index(i0 + li - 2, g.nx, g.perx);
    const int gj = halo_index(j0 + lj - 2, g.ny, g.pery);
    dst[li][lj] = pk[(long long)gi * g.ny + gj];
  }
}

template <int ACTX, int WID>
__device__ __forceinline__ double fast_K(const double (*A)[WID], int r, int c, double ax, double ay,
                                         double cK) {
  double t = ay * (A[r][c - 1] + A[r][c + 1]);
  if (ACTX) t = fma(ax, A[r - 1][c] + A[r + 1][c], t);
  return fma(cK, A[r][c], -t);
}

template <int ACTX>
__global__ void __launch_bounds__(TI * TJ, 2) k_AAt(Geom g, int kc, const double* __restrict__ p,
                                                    double* __restrict__ q, double* partials,
                                                    DevScalars* sc, int mode) {
  if (mode == 1 && sc->cg_done) return;
  __shared__ double P[2][H2I][H2J];
  __shared__ double XM[H1I][H1J];
  __shared__ double KP[TI][TJ];
  const int tj = threadIdx.x, ti = threadIdx.y;
  const int j0 = blockIdx.x * TJ, i0 = blockIdx.y * TI;
  const int k0 = blockIdx.z * kc;
  const int k1 = min(g.nt, k0 + kc);
  const int gi = i0 + ti, gj = j0 + tj;
  const bool own = gi < g.nx && gj < g.ny;
  const double ax = ACTX ? g.ax : 0.0, ay = g.ay, cK = 2.0 * (ax + ay);
  const double nax = g.nu * ax, nay = g.nu * ay, ncK = g.nu * cK;
  // xm halo slots that lie outside a Neumann axis (rebuilt from their mirrors)
  const bool ghost_x = ACTX && !g.perx && (i0 == 0 || i0 + TI >= g.nx);
  const bool ghost_y = !g.pery && (j0 == 0 || j0 + TJ >= g.ny);
  const bool ghosts = ghost_x || ghost_y;
  const int tid = tj + TJ * ti;

  int cur = 0;
  load_plane_h2(g, p, k0, i0, j0, P[cur]);
  double xprev = 0.0;
  if (k0 > 0) {
    load_plane_h2(g, p, k0 - 1, i0, j0, P[cur ^ 1]);
    __syncthreads();
    if (own)
      xprev = fast_K<ACTX, H2J>(P[cur ^ 1], ti + 2, tj + 2, nax, nay, ncK) +
              (P[cur ^ 1][ti + 2][tj + 2] - P[cur][ti + 2][tj + 2]) * g.idt;
    __syncthreads();
  }
  double acc = 0.0;
  for (int k = k0; k < k1; ++k) {
    load_plane_h2(g, p, k + 1, i0, j0, P[cur ^ 1]);
    __syncthreads();
    const double (*Pk)[H2J] = P[cur];
    const double (*Pn)[H2J] = P[cur ^ 1];
    // One FP64 sequence for every slot (no divergent paths): K p, then xm.
    for (int s = tid; s < H1I * H1J; s += TI * TJ) {
      const int li = s / H1J, lj = s % H1J;
      const double kp = fast_K<ACTX, H2J>(Pk, li + 1, lj + 1, ax, ay, cK);
      XM[li][lj] = fma(g.nu, kp, (Pk[li + 1][lj + 1] - Pn[li + 1][lj + 1]) * g.idt);
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
          // mirror slot is inside the domain (read-only here: distinct from ghosts)
          XM[li][lj] = XM[mi][mj];
        }
      }
      __syncthreads();
    }
    if (own) {
      const double c = XM[ti + 1][tj + 1];
      const double nKxm = fast_K<ACTX, H1J>(XM, ti + 1, tj + 1, nax, nay, ncK);
      const double val = fma(2.0, KP[ti][tj], fma(c - xprev, g.idt, nKxm));
      xprev = c;
      const long long e = (long long)k * g.S + (long long)gi * g.ny + gj;
      q[e] = val;
      acc = fma(val, Pk[ti + 2][tj + 2], acc);
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

// The same fused stencil in double-float arithmetic (df64.cuh): p is split into
// FP32 pairs as it is staged, every stencil operation runs on FP32 pairs, and q
// is rebuilt in FP64 (one FP64 add per point) together with the FP64 p.q.
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

void launch_AAt(const Geom& g, const double* p, double* q, double* partials, DevScalars* sc,
                int mode, cudaStream_t s, int df64) {
  const int kc = aat_chunk(g);
  dim3 grid((g.ny + TJ - 1) / TJ, (g.nx + TI - 1) / TI, (g.nt + kc - 1) / kc);
  dim3 block(TJ, TI);
  if (df64) {
    if (g.actx)
      k_AAt_df<1><<<grid, block, 0, s>>>(g, kc, p, q, partials, sc, mode);
    else
      k_AAt_df<0><<<grid, block, 0, s>>>(g, kc, p, q, partials, sc, mode);
    return;
  }
  if (g.actx)
    k_AAt<1><<<grid, block, 0, s>>>(g, kc, p, q, partials, sc, mode);
  else
    k_AAt<0><<<grid, block, 0, s>>>(g, kc, p, q, partials, sc, mode);
}

}  // namespace mfg
