// The parallel-in-time preconditioner P of Sec. 4 (eq. prec), applied through
// its fully diagonalised form eq. pstrec:
//   P = (V^T (x) H^T (x) G^T) (I (x) Lambda_1 + Lambda_t (x) Lambda_2) (V (x) H (x) G),
// i.e. Alg. 1 with Alg. 2 in place of its per-time-step solve.
//
// Transforms (all real and orthonormal, so the inverse is the transpose):
//   time  V: DCT-VIII for l = 1, DST-I for l = 2 (Sec. 4.1, eigenvalues eq. eigs)
//   space H, G: periodic axis -> discrete Hartley transform, a real orthonormal
//         eigenbasis of the circulant Laplacian (same eigenvalues
//         2 - 2cos(2 pi v/N) as the DFT of Alg. 2); Neumann axis -> DCT-II
//         (eigenvalues 2 - 2cos(pi v/N), Alg. 2).
//   Lambda_1 = nu^2 D^2 + 2 D, Lambda_2 = (nu D + 1/dt)/dt (eq. lambda1, lambda2)
//   with D the tiled spatial eigenvalues of Alg. 2; the per-frequency
//   divisor S = Lambda_1 + lambda_k Lambda_2 (Alg. 2) is formed on
//   the fly, never stored as an n-sized table.
//
// Passes over the data (ping-pong work buffers, 10n words in total):
//   y-forward, x-forward, [time forward, divide by S, time inverse] fused,
//   x-inverse, y-inverse.  A spatial pass is an FFT (k_fft.cu) when the axis
//   length is a power of two from 8 to 512, otherwise a small dense matrix
//   applied along the axis (a SIMT GEMM with the transform matrix on the
//   left); the time pass keeps a strip of all N_t planes in shared memory.
#include <cmath>
#include <vector>

#include "mfg_internal.cuh"

namespace mfg {

// ---------------------------------------------------------------- tables --
static void axis_basis(int N, int periodic, std::vector<double>& H, std::vector<double>& lam) {
  H.assign((size_t)N * N, 0.0);
  lam.assign(N, 0.0);
  const double pi = 3.14159265358979323846;
  if (N == 1) {
    H[0] = 1.0;
    return;
  }
  for (int a = 0; a < N; ++a) {
    if (periodic) {
      lam[a] = 2.0 - 2.0 * std::cos(2.0 * pi * a / N);
      for (int b = 0; b < N; ++b) {
        const double th = 2.0 * pi * (double)((long long)a * b % N) / N;
        H[(size_t)a * N + b] = (std::cos(th) + std::sin(th)) / std::sqrt((double)N);
      }
    } else {
      lam[a] = 2.0 - 2.0 * std::cos(pi * a / N);
      const double ca = a == 0 ? std::sqrt(1.0 / N) : std::sqrt(2.0 / N);
      for (int b = 0; b < N; ++b) H[(size_t)a * N + b] = ca * std::cos(pi * a * (2.0 * b + 1.0) / (2.0 * N));
    }
  }
}

static void time_basis(int N, int l, std::vector<double>& V, std::vector<double>& lam) {
  V.assign((size_t)N * N, 0.0);
  lam.assign(N, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < N; ++k) {
    if (l == 1) {
      lam[k] = 2.0 - 2.0 * std::cos(pi * (k + 0.5) / (N + 0.5));
      for (int j = 0; j < N; ++j)
        V[(size_t)k * N + j] = 2.0 / std::sqrt(2.0 * N + 1.0) *
                               std::cos(pi * (2.0 * k + 1.0) * (2.0 * j + 1.0) / (2.0 * (2.0 * N + 1.0)));
    } else {
      lam[k] = 2.0 - 2.0 * std::cos(pi * (k + 1.0) / (N + 1.0));
      for (int j = 0; j < N; ++j)
        V[(size_t)k * N + j] = std::sqrt(2.0 / (N + 1.0)) * std::sin(pi * (j + 1.0) * (k + 1.0) / (N + 1.0));
    }
  }
}

// max |M M^T - I|: orthonormality guard on the host tables.
static double ortho_defect(const std::vector<double>& M, int N) {
  double worst = 0.0;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      double s = 0.0;
      for (int t = 0; t < N; ++t) s += M[(size_t)a * N + t] * M[(size_t)b * N + t];
      worst = std::fmax(worst, std::fabs(s - (a == b ? 1.0 : 0.0)));
    }
  return worst;
}

template <typename T>
static T* upload(const std::vector<double>& h, std::string* err) {
  std::vector<T> tmp(h.begin(), h.end());
  T* d = nullptr;
  if (cudaMalloc(&d, sizeof(T) * tmp.size()) != cudaSuccess) {
    *err = "cudaMalloc failed for preconditioner tables";
    return nullptr;
  }
  if (cudaMemcpy(d, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = "cudaMemcpy failed for preconditioner tables";
    cudaFree(d);
    return nullptr;
  }
  return d;
}

int build_prec_tables(const mfg_problem& p, const Geom& g, PrecTables* t, std::string* err) {
  *t = PrecTables{};
  t->nx = g.nx;
  t->ny = g.ny;
  t->nt = g.nt;
  std::vector<double> Hx, lx, Hy, ly, V, lt;
  axis_basis(g.nx, g.perx, Hx, lx);
  axis_basis(g.ny, g.pery, Hy, ly);
  time_basis(g.nt, p.l == 0 ? 2 : p.l, V, lt);  // l = 0 has no time transform (unused table)
  const double dx_defect = std::fmax(ortho_defect(Hx, g.nx), ortho_defect(Hy, g.ny));
  const double dt_defect = ortho_defect(V, g.nt);
  if (dx_defect > 1e-10 || dt_defect > 1e-10) {
    *err = "transform tables failed the orthonormality check";
    return MFG_ERR_INVALID_ARG;
  }
  double asym = 0.0;
  for (int a = 0; a < g.nt; ++a)
    for (int b = 0; b < g.nt; ++b) asym = std::fmax(asym, std::fabs(V[(size_t)a * g.nt + b] - V[(size_t)b * g.nt + a]));
  if (asym > 1e-12) {
    *err = "time transform table is not symmetric";
    return MFG_ERR_INVALID_ARG;
  }
  std::vector<double> L1((size_t)g.S), L2((size_t)g.S);
  if (p.l == 0) {
    // Exact variant (P = AAt): per spatial mode with Laplacian eigenvalue kappa,
    // the block of eq. largeA is the SPD tridiagonal matrix with diagonal
    // (C, C + 1/dt^2, ...), C = L^2 + 2 kappa, L = nu kappa + 1/dt, and
    // off-diagonal -L/dt.  Its Thomas factors depend only on the mode, so they
    // are formed once here: c_k = off/den_k and 1/den_k, den_k = diag_k - off c_{k-1}.
    std::vector<double> cf((size_t)g.n), idn((size_t)g.n), off((size_t)g.S);
    const double dtv = 1.0 / g.idt;
    for (int a = 0; a < g.nx; ++a)
      for (int b = 0; b < g.ny; ++b) {
        const size_t sidx = (size_t)a * g.ny + b;
        const double kap = lx[a] * g.ax + ly[b] * g.ay;
        const double Ls = g.nu * kap + 1.0 / dtv;
        const double Cs = Ls * Ls + 2.0 * kap;
        const double o = -Ls / dtv;
        off[sidx] = o;
        double cprev = 0.0;
        for (int k = 0; k < g.nt; ++k) {
          const double diag = Cs + (k >= 1 ? 1.0 / (dtv * dtv) : 0.0);
          const double den = diag - (k >= 1 ? o * cprev : 0.0);
          const size_t e = (size_t)k * g.S + sidx;
          idn[e] = 1.0 / den;
          cprev = o / den;
          cf[e] = cprev;
        }
      }
    t->thc64 = upload<double>(cf, err);
    t->thd64 = upload<double>(idn, err);
    t->tho64 = upload<double>(off, err);
    t->thc32 = upload<float>(cf, err);
    t->thd32 = upload<float>(idn, err);
    t->tho32 = upload<float>(off, err);
    if (!t->thc64 || !t->thd64 || !t->tho64 || !t->thc32 || !t->thd32 || !t->tho32) {
      free_prec_tables(t);
      return MFG_ERR_CUDA;
    }
  }
  const double dtv = 1.0 / g.idt, nu = g.nu;
  for (int a = 0; a < g.nx; ++a)
    for (int b = 0; b < g.ny; ++b) {
      const double D = lx[a] * g.ax + ly[b] * g.ay;
      L1[(size_t)a * g.ny + b] = nu * nu * D * D + 2.0 * D;
      L2[(size_t)a * g.ny + b] = (nu * D + 1.0 / dtv) / dtv;
    }
  t->Hx64 = upload<double>(Hx, err);
  t->Hy64 = upload<double>(Hy, err);
  t->Vt64 = upload<double>(V, err);
  t->lamt64 = upload<double>(lt, err);
  t->L1_64 = upload<double>(L1, err);
  t->L2_64 = upload<double>(L2, err);
  t->Hx32 = upload<float>(Hx, err);
  t->Hy32 = upload<float>(Hy, err);
  t->Vt32 = upload<float>(V, err);
  t->lamt32 = upload<float>(lt, err);
  t->L1_32 = upload<float>(L1, err);
  t->L2_32 = upload<float>(L2, err);
  // FFT twiddles: tw[m] = (cos, sin)(2 pi m/N), dct[k] = (cos, sin)(pi k/(2N)).
  auto fft_tables = [&](int N, double** tw64, float** tw32, double** dc64, float** dc32) {
    if (!fft_supported(N)) return true;
    const double pi = 3.14159265358979323846;
    std::vector<double> tw((size_t)N), dc((size_t)2 * N);
    for (int m = 0; m < N / 2; ++m) {
      tw[2 * m] = std::cos(2.0 * pi * m / N);
      tw[2 * m + 1] = std::sin(2.0 * pi * m / N);
    }
    for (int k = 0; k < N; ++k) {
      dc[2 * k] = std::cos(pi * k / (2.0 * N));
      dc[2 * k + 1] = std::sin(pi * k / (2.0 * N));
    }
    *tw64 = upload<double>(tw, err);
    *tw32 = upload<float>(tw, err);
    *dc64 = upload<double>(dc, err);
    *dc32 = upload<float>(dc, err);
    return *tw64 && *tw32 && *dc64 && *dc32;
  };
  const bool fft_ok = (g.nx == 1 || fft_tables(g.nx, &t->twx64, &t->twx32, &t->dctx64, &t->dctx32)) &&
                      fft_tables(g.ny, &t->twy64, &t->twy32, &t->dcty64, &t->dcty32);
  if (!fft_ok || !t->Hx64 || !t->Hy64 || !t->Vt64 || !t->lamt64 || !t->L1_64 || !t->L2_64 || !t->Hx32 ||
      !t->Hy32 || !t->Vt32 || !t->lamt32 || !t->L1_32 || !t->L2_32) {
    free_prec_tables(t);
    return MFG_ERR_CUDA;
  }
  if (p.nu_field != nullptr) {
    const int rc = build_band_tables(p, g, lt.data(), t, err);
    if (rc != MFG_OK) {
      free_prec_tables(t);
      return rc;
    }
  }
  return MFG_OK;
}

void free_prec_tables(PrecTables* t) {
  void* ptrs[] = {t->Hx64, t->Hy64, t->Vt64, t->lamt64, t->L1_64, t->L2_64, t->Hx32, t->Hy32,
                  t->Vt32, t->lamt32, t->L1_32, t->L2_32, t->twx64, t->twx32, t->dctx64, t->dctx32,
                  t->twy64, t->twy32, t->dcty64, t->dcty32, t->thc64, t->thd64, t->tho64,
                  t->thc32, t->thd32, t->tho32, t->kfx, t->kfy, t->band_perm, t->bandc64,
                  t->bandr64, t->bandc32, t->bandr32};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  *t = PrecTables{};
}

// ------------------------------------------------------- axis transform --
// out(a, col) = sum_b M(a, b) in(b, col), M(a, b) = trans ? M[b*N + a] : M[a*N + b],
// where column col = (o, i) addresses in[(o*N + b)*inner + i].  CONTIG: the
// transformed axis is the contiguous one (inner == 1).
constexpr int BM = 64, BN = 64, BK = 16;

template <typename TI, typename T, typename TO, bool CONTIG>
__global__ void __launch_bounds__(256) k_axis(const TI* __restrict__ in, TO* __restrict__ out,
                                              const T* __restrict__ M, int N, long long inner,
                                              long long ncols, int trans, const DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tr = CONTIG ? (tid & 15) : (tid >> 4);
  const int tc = CONTIG ? (tid >> 4) : (tid & 15);
  const int a0 = blockIdx.y * BM;
  const long long c0 = (long long)blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);

  for (int b0 = 0; b0 < N; b0 += BK) {
    // A tile: As[bb][aa] = M(a0+aa, b0+bb)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s = tid + 256 * q;
      int aa, bb;
      if (trans) { aa = s % BM; bb = s / BM; } else { bb = s % BK; aa = s / BK; }
      const int a = a0 + aa, b = b0 + bb;
      T val = T(0);
      if (a < N && b < N) val = trans ? M[(long long)b * N + a] : M[(long long)a * N + b];
      As[bb][aa] = val;
    }
    // B tile: Bs[bb][cc] = in(b0+bb, c0+cc)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s = tid + 256 * q;
      int bb, cc;
      if (CONTIG) { bb = s % BK; cc = s / BK; } else { cc = s % BN; bb = s / BN; }
      const int b = b0 + bb;
      const long long col = c0 + cc;
      T val = T(0);
      if (b < N && col < ncols) {
        const long long o = col / inner, i = col - o * inner;
        val = (T)in[(o * N + b) * inner + i];
      }
      Bs[bb][cc] = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = As[kk][tr + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) bv[v] = Bs[kk][tc + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = a0 + tr + 16 * u;
    if (a >= N) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long col = c0 + tc + 16 * v;
      if (col >= ncols) continue;
      const long long o = col / inner, i = col - o * inner;
      out[(o * N + a) * inner + i] = (TO)acc[u][v];
    }
  }
}

template <typename TI, typename T, typename TO>
static void axis_pass(const TI* in, TO* out, const T* M, int N, long long inner, long long outer,
                      int trans, const DevScalars* sc, cudaStream_t s) {
  const long long ncols = inner * outer;
  dim3 grid((unsigned)((ncols + BN - 1) / BN), (N + BM - 1) / BM);
  if (inner == 1)
    k_axis<TI, T, TO, true><<<grid, 256, 0, s>>>(in, out, M, N, inner, ncols, trans, sc);
  else
    k_axis<TI, T, TO, false><<<grid, 256, 0, s>>>(in, out, M, N, inner, ncols, trans, sc);
}

// ------------------------------------------------------ fused time pass --
// For a strip of TSW spatial modes: Y = V X (time forward), Y /= S(k, s),
// out = V^T Y (time inverse).  One strip buffer (N_t x TSW) is reused for X
// and then Y; V is streamed through shared memory in 16-column chunks.
constexpr int TSW = 32, TCH = 16, TU = kMaxNt / 8;

template <typename T>
__global__ void __launch_bounds__(256) k_time(const T* __restrict__ in, T* __restrict__ out,
                                              const T* __restrict__ V, const T* __restrict__ lamt,
                                              const T* __restrict__ L1, const T* __restrict__ L2,
                                              int nt, int S, const DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  extern __shared__ unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);   // [nt][TSW]
  T* Vs = X + (size_t)nt * TSW;            // [nt][TCH]
  const int tid = threadIdx.x, c = tid % TSW, r0 = tid / TSW;
  const int s0 = blockIdx.x * TSW;
  const int sc_ = s0 + c;
  for (int q = tid; q < nt * TSW; q += 256) {
    const int k = q / TSW, cc = q % TSW;
    X[q] = (s0 + cc < S) ? in[(long long)k * S + s0 + cc] : T(0);
  }
  const int nu_ = (nt + 7) / 8;
  T acc[TU];
#pragma unroll
  for (int u = 0; u < TU; ++u) acc[u] = T(0);
  // Y = V X
  for (int b0 = 0; b0 < nt; b0 += TCH) {
    __syncthreads();
    for (int q = tid; q < nt * TCH; q += 256) {
      const int a = q / TCH, bb = q % TCH;
      Vs[q] = (b0 + bb < nt) ? V[(long long)a * nt + b0 + bb] : T(0);
    }
    __syncthreads();
    const int bmax = min(TCH, nt - b0);
    for (int bb = 0; bb < bmax; ++bb) {
      const T xb = X[(b0 + bb) * TSW + c];
#pragma unroll
      for (int u = 0; u < TU; ++u)
        if (u < nu_) {
          const int a = r0 + 8 * u;
          if (a < nt) acc[u] = fma(Vs[a * TCH + bb], xb, acc[u]);
        }
    }
  }
  __syncthreads();
  // divide by S(k, s) = Lambda_1(s) + lambda_k Lambda_2(s); overwrite X with Y
  const T l1 = sc_ < S ? L1[sc_] : T(1), l2 = sc_ < S ? L2[sc_] : T(0);
#pragma unroll
  for (int u = 0; u < TU; ++u)
    if (u < nu_) {
      const int a = r0 + 8 * u;
      if (a < nt) X[a * TSW + c] = acc[u] / (l1 + lamt[a] * l2);
      acc[u] = T(0);
    }
  // out = V^T Y
  for (int b0 = 0; b0 < nt; b0 += TCH) {
    __syncthreads();
    for (int q = tid; q < nt * TCH; q += 256) {
      const int a = q / TCH, bb = q % TCH;
      Vs[q] = (b0 + bb < nt) ? V[(long long)(b0 + bb) * nt + a] : T(0);
    }
    __syncthreads();
    const int bmax = min(TCH, nt - b0);
    for (int bb = 0; bb < bmax; ++bb) {
      const T yb = X[(b0 + bb) * TSW + c];
#pragma unroll
      for (int u = 0; u < TU; ++u)
        if (u < nu_) {
          const int a = r0 + 8 * u;
          if (a < nt) acc[u] = fma(Vs[a * TCH + bb], yb, acc[u]);
        }
    }
  }
  if (sc_ < S) {
#pragma unroll
    for (int u = 0; u < TU; ++u)
      if (u < nu_) {
        const int a = r0 + 8 * u;
        if (a < nt) out[(long long)a * S + sc_] = acc[u];
      }
  }
}

// Fixed-N_t time pass: the whole (symmetric, orthonormal) time matrix V sits in
// shared memory next to an N_t x TW strip; each thread owns an RM x RN register
// tile, so one pass over b costs RM + RN shared loads for RM * RN FMAs.  Both
// DCT-VIII and DST-I are symmetric (V = V^T, checked on the host), so rows of V
// serve the forward and the inverse product.
template <typename T, int NT>
struct TimeShape {
  static constexpr int TW = 32;                           // strip width (spatial modes)
  static constexpr int RN = 2;                            // columns per thread
  static constexpr int CG = TW / RN;                      // column groups
  static constexpr int RG = 256 / CG;                     // row groups
  static constexpr int RM = NT / RG;                      // rows per thread
  static constexpr size_t smem = sizeof(T) * ((size_t)NT * NT + (size_t)NT * TW);
};

// K consecutive shared-memory values with the widest aligned vector loads.
template <int K>
__device__ __forceinline__ void lds_vec(const float* p, float (&o)[K]) {
  if constexpr (K % 4 == 0) {
#pragma unroll
    for (int q = 0; q < K; q += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + q);
      o[q] = v.x; o[q + 1] = v.y; o[q + 2] = v.z; o[q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < K; ++q) o[q] = p[q];
  }
}
template <int K>
__device__ __forceinline__ void lds_vec(const double* p, double (&o)[K]) {
  if constexpr (K % 2 == 0) {
#pragma unroll
    for (int q = 0; q < K; q += 2) {
      const double2 v = *reinterpret_cast<const double2*>(p + q);
      o[q] = v.x; o[q + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < K; ++q) o[q] = p[q];
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(256) k_time_fast(const T* __restrict__ in, T* __restrict__ out,
                                                   const T* __restrict__ V, const T* __restrict__ lamt,
                                                   const T* __restrict__ L1, const T* __restrict__ L2,
                                                   int S, const DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  using Sh = TimeShape<T, NT>;
  constexpr int TW = Sh::TW, RN = Sh::RN, CG = Sh::CG, RM = Sh::RM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);  // [NT][NT], loaded once per block
  T* X = Vs + NT * NT;                      // [NT][TW]
  const int tid = threadIdx.x;
  const int cg = tid % CG, rg = tid / CG;
  const int r0 = rg * RM;  // this thread's rows r0 .. r0 + RM - 1
  for (int q = tid; q < NT * NT; q += 256) Vs[q] = V[q];
  T lam[RM];
#pragma unroll
  for (int u = 0; u < RM; ++u) lam[u] = lamt[r0 + u];
  const int nstrips = (S + TW - 1) / TW;
  // the block walks strips of TW spatial modes, reusing V from shared memory
  for (int strip = blockIdx.x; strip < nstrips; strip += gridDim.x) {
    const int s0 = strip * TW;
    __syncthreads();  // previous strip done with X (and V loaded on the first pass)
    for (int q = tid; q < NT * TW; q += 256) {
      const int k = q / TW, c = q % TW;
      X[q] = (s0 + c < S) ? in[(long long)k * S + s0 + c] : T(0);
    }
    __syncthreads();
    T acc[RM][RN];
#pragma unroll
    for (int u = 0; u < RM; ++u)
#pragma unroll
      for (int v = 0; v < RN; ++v) acc[u][v] = T(0);
    // Y = V X: row r uses V[r][b] = V[b][r] (symmetric V), contiguous in r
#pragma unroll 4
    for (int b = 0; b < NT; ++b) {
      T xv[RN], vv[RM];
      lds_vec<RN>(X + b * TW + cg * RN, xv);
      lds_vec<RM>(Vs + b * NT + r0, vv);
#pragma unroll
      for (int u = 0; u < RM; ++u)
#pragma unroll
        for (int v = 0; v < RN; ++v) acc[u][v] = fma(vv[u], xv[v], acc[u][v]);
    }
    __syncthreads();
    // divide by S(k, s) = Lambda_1(s) + lambda_k Lambda_2(s); Y overwrites X
#pragma unroll
    for (int v = 0; v < RN; ++v) {
      const int c = cg * RN + v;
      const int s = s0 + c;
      const T l1 = s < S ? L1[s] : T(1), l2 = s < S ? L2[s] : T(0);
#pragma unroll
      for (int u = 0; u < RM; ++u) {
        X[(r0 + u) * TW + c] = acc[u][v] / (l1 + lam[u] * l2);
        acc[u][v] = T(0);
      }
    }
    __syncthreads();
    // out = V^T Y: out[a][c] = sum_b V[b][a] Y[b][c]
#pragma unroll 4
    for (int b = 0; b < NT; ++b) {
      T yv[RN], vv[RM];
      lds_vec<RN>(X + b * TW + cg * RN, yv);
      lds_vec<RM>(Vs + b * NT + r0, vv);
#pragma unroll
      for (int u = 0; u < RM; ++u)
#pragma unroll
        for (int v = 0; v < RN; ++v) acc[u][v] = fma(vv[u], yv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < RM; ++u) {
      const int r = r0 + u;
#pragma unroll
      for (int v = 0; v < RN; ++v) {
        const int s = s0 + cg * RN + v;
        if (s < S) out[(long long)r * S + s] = acc[u][v];
      }
    }
  }
}

template <typename T, int NT>
static void launch_time_fast(const T* in, T* out, const T* V, const T* lamt, const T* L1, const T* L2,
                             int S, const DevScalars* sc, cudaStream_t s) {
  using Sh = TimeShape<T, NT>;
  // enough blocks to fill the GPU (several resident per SM); each walks strips
  const int nstrips = (S + Sh::TW - 1) / Sh::TW;
  const int blocks = nstrips < 152 * 4 ? nstrips : 152 * 4;
  k_time_fast<T, NT><<<blocks, 256, Sh::smem, s>>>(in, out, V, lamt, L1, L2, S, sc);
}

// Exact time solve of the l = 0 variant: per spatial mode s, the tridiagonal
// system of eq. largeA in time by Thomas elimination with the precomputed
// factors (forward sweep into `out`, then back substitution in place).  One
// thread per mode; loads at a fixed k are contiguous across the threads.
template <typename T>
__global__ void __launch_bounds__(256) k_thomas(const T* __restrict__ in, T* __restrict__ out,
                                                const T* __restrict__ cf, const T* __restrict__ idn,
                                                const T* __restrict__ off, int nt, int S,
                                                const DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const T o = off[s];
    T d = T(0);
#pragma unroll 8
    for (int k = 0; k < nt; ++k) {
      const long long e = (long long)k * S + s;
      d = (in[e] - o * d) * idn[e];
      out[e] = d;
    }
    T x = d;
#pragma unroll 8
    for (int k = nt - 2; k >= 0; --k) {
      const long long e = (long long)k * S + s;
      x = out[e] - cf[e] * x;
      out[e] = x;
    }
  }
}

template <typename T>
static size_t time_smem(int nt) { return sizeof(T) * (size_t)nt * (TSW + TCH); }

template <typename T>
static void time_pass(const T* in, T* out, const T* V, const T* lamt, const T* L1, const T* L2,
                      int nt, int S, const DevScalars* sc, cudaStream_t s) {
  if (nt == 32) return launch_time_fast<T, 32>(in, out, V, lamt, L1, L2, S, sc, s);
  if (nt == 64) return launch_time_fast<T, 64>(in, out, V, lamt, L1, L2, S, sc, s);
  if (nt == 128) return launch_time_fast<T, 128>(in, out, V, lamt, L1, L2, S, sc, s);
  const size_t sm = time_smem<T>(nt);
  k_time<T><<<(S + TSW - 1) / TSW, 256, sm, s>>>(in, out, V, lamt, L1, L2, nt, S, sc);
}

template <typename T>
static void precond_typed(const Geom& g, const T* Hx, const T* Hy, const T* V, const T* lamt,
                          const T* L1, const T* L2, const T* twx, const T* dctx, const T* twy,
                          const T* dcty, const T* thc, const T* thd, const T* tho,
                          const double* r, double* z, T* w0, T* w1,
                          const DevScalars* sc, cudaStream_t s, const PcgDot* dot,
                          const PcgZr* zr, bool tc = false) {
  const long long S = g.S, n = g.n;
  const bool fy = g.fft_y && twy != nullptr && fft_supported(g.ny);
  const bool fx = g.fft_x && twx != nullptr && fft_supported(g.nx);
  // y forward: axis length ny, contiguous
  if (fy) {
    fft_y_forward<T>(g.ny, g.pery, r, w0, twy, dcty, n / g.ny, sc, s, zr);
  } else {
    if (zr) launch_update_zr(n, zr->z, zr->r, zr->p, zr->q, zr->partials, zr->sc, s, g.vec_blocks);
    axis_pass<double, T, T>(r, w0, Hy, g.ny, 1, n / g.ny, 0, sc, s);
  }
  T* a = w0;
  T* b = w1;
  if (g.nx > 1) {
    if (fx)
      fft_x<T>(g.nx, g.perx, 0, a, b, twx, dctx, g.ny, (long long)g.nt, sc, s);
    else
      axis_pass<T, T, T>(a, b, Hx, g.nx, g.ny, (long long)g.nt, 0, sc, s);
    T* t = a; a = b; b = t;
  }
  if (thc != nullptr) {
    k_thomas<T><<<(int)((S + 255) / 256), 256, 0, s>>>(a, b, thc, thd, tho, g.nt, (int)S, sc);
  } else if constexpr (sizeof(T) == 4) {
    if (tc && !g.time_simt && time_tc_supported(g.nt))
      launch_time_tc(a, b, V, lamt, L1, L2, g.nt, (int)S, sc, s);
    else
      time_pass<T>(a, b, V, lamt, L1, L2, g.nt, (int)S, sc, s);
  } else {
    time_pass<T>(a, b, V, lamt, L1, L2, g.nt, (int)S, sc, s);
  }
  { T* t = a; a = b; b = t; }
  if (g.nx > 1) {
    if (fx)
      fft_x<T>(g.nx, g.perx, 1, a, b, twx, dctx, g.ny, (long long)g.nt, sc, s);
    else
      axis_pass<T, T, T>(a, b, Hx, g.nx, g.ny, (long long)g.nt, 1, sc, s);
    T* t = a; a = b; b = t;
  }
  if (fy) {
    fft_y_inverse<T>(g.ny, g.pery, a, z, twy, dcty, n / g.ny, sc, s, dot);
  } else {
    axis_pass<T, T, double>(a, z, Hy, g.ny, 1, n / g.ny, 1, sc, s);
    if (dot) launch_dot_beta(n, dot->r, z, dot->q, dot->flex, dot->partials, dot->sc, s, g.vec_blocks);
  }
}

void launch_precond(const Geom& g, const PrecTables& t, int precision, const double* r, double* z,
                    double* work64, float* work32, const DevScalars* sc, cudaStream_t s,
                    const PcgDot* dot, const PcgZr* zr) {
  if (t.band_w > 0) {  // viscosity field: time transforms around banded per-frequency solves
    if (zr) launch_update_zr(g.n, zr->z, zr->r, zr->p, zr->q, zr->partials, zr->sc, s, g.vec_blocks);
    launch_precond_band(g, t, precision, r, z, work64, work32, sc, s);
    if (dot) launch_dot_beta(g.n, dot->r, z, dot->q, dot->flex, dot->partials, dot->sc, s, g.vec_blocks);
    return;
  }
  if (precision == MFG_MIXED || precision == MFG_MIXED_DF || precision == MFG_MIXED_TC)
    precond_typed<float>(g, t.Hx32, t.Hy32, t.Vt32, t.lamt32, t.L1_32, t.L2_32, t.twx32, t.dctx32,
                         t.twy32, t.dcty32, t.thc32, t.thd32, t.tho32, r, z, work32, work32 + g.n,
                         sc, s, dot, zr, precision == MFG_MIXED_TC);
  else
    precond_typed<double>(g, t.Hx64, t.Hy64, t.Vt64, t.lamt64, t.L1_64, t.L2_64, t.twx64, t.dctx64,
                          t.twy64, t.dcty64, t.thc64, t.thd64, t.tho64, r, z, work64, work64 + g.n,
                          sc, s, dot, zr);
}

int precond_kernel_count(const Geom& g) { return g.kfy != nullptr ? 4 : (g.nx > 1 ? 5 : 3); }

// Kernels of a preconditioner apply that also runs the PCG update and dot products.
int precond_step_kernel_count(const Geom& g, const PrecTables& t) {
  if (t.band_w > 0) return 4 + 2;
  const bool fused = g.fft_y && t.twy32 != nullptr && fft_supported(g.ny);
  return precond_kernel_count(g) + (fused ? 0 : 2);
}

// Opt-in shared memory for the time pass; called once per device before any
// launch or stream capture.
int precond_configure() {
  cudaError_t e1 = cudaFuncSetAttribute(k_time<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)time_smem<double>(kMaxNt));
  cudaError_t e2 = cudaFuncSetAttribute(k_time<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)time_smem<float>(kMaxNt));
  int bad = (e1 != cudaSuccess) || (e2 != cudaSuccess);
#define MFG_TF_ATTR(T, NT)                                                                    \
  bad |= cudaFuncSetAttribute(k_time_fast<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                              (int)TimeShape<T, NT>::smem) != cudaSuccess;
  MFG_TF_ATTR(float, 32) MFG_TF_ATTR(float, 64) MFG_TF_ATTR(float, 128)
  MFG_TF_ATTR(double, 32) MFG_TF_ATTR(double, 64) MFG_TF_ATTR(double, 128)
#undef MFG_TF_ATTR
  bad |= fft_configure() != MFG_OK;
  bad |= band_configure() != MFG_OK;
  bad |= prox_configure() != MFG_OK;
  bad |= time_tc_configure() != MFG_OK;
  return bad ? MFG_ERR_CUDA : MFG_OK;
}

}  // namespace mfg
