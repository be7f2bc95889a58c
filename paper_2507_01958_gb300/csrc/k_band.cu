// Viscosity fields nu(x): Alg. 1 of Sec. 4 with an exact solve of every
// per-frequency system, the LU option the paper names for the per-time-step
// systems (Sec. 4.1, after Alg. 1).
//
// With K_nu = sum_axes D^1 diag(nu_face) (D^1)^T / dx^2 in place of nu K, the
// blocks of eq. prec are C_hat = K_nu^2 + B B^T = K_nu^2 + 2K (eq. precstead)
// and L_hat = (K_nu + I/dt)/dt.  The time transform V (DCT-VIII or DST-I,
// symmetric and orthonormal) still block-diagonalises P:
//   P^{-1} r = V diag_k (C_hat + lambda_k L_hat)^{-1} V r,
// but the spatial blocks no longer share the Laplacian's eigenbasis.  Each
// M_k = C_hat + lambda_k L_hat is SPD and banded once the points are ordered
// axis by axis (a periodic axis folded 0, N-1, 1, N-2, ... so that wrapped
// neighbours stay close), so it is factored M_k = L_k L_k^T by banded
// Cholesky on the host in FP64, once per plan.  An apply is
//   time forward (scatter to band order) -> L y = b -> L^T x = y -> time
//   inverse (gather from band order).
// The substitutions are sequential along the band: one CTA per frequency
// walks its S points in blocks of up to 32 (a warp-shuffle triangular solve,
// then a block update of the next w partial sums, held in a circular window
// in shared memory); the factor rows, contiguous in memory in the order they
// are used, stream through a ring of shared-memory stages filled by cp.async
// several blocks ahead, so the loads never wait on the dependency chain.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "mfg_internal.cuh"

namespace mfg {

namespace {

constexpr int kBandRing = 5;           // shared-memory stages of factor rows
constexpr int kBandStageBytes = 40 * 1024;
constexpr int kBandMaxW = 4096;
constexpr double kBandMaxBytes = 64.0 * 1024 * 1024 * 1024;

// rank of node i along an axis: identity on a Neumann axis, folded on a
// periodic one (neighbours i, i+-1 and i+-2 mod N land at most 2 and 4 apart)
std::vector<int> axis_rank(int N, int per) {
  std::vector<int> r((size_t)N);
  for (int i = 0; i < N; ++i) r[(size_t)i] = (!per) ? i : (2 * i < N ? 2 * i : 2 * (N - 1 - i) + 1);
  return r;
}

// Sparse row with a handful of entries (K_nu^2 has at most 13 per row).
struct Row {
  int col[32];
  double val[32];
  int n = 0;
  void add(int c, double v) {
    for (int q = 0; q < n; ++q)
      if (col[q] == c) {
        val[q] += v;
        return;
      }
    col[n] = c;
    val[n] = v;
    ++n;
  }
};

// Row a of the 5-point operator sum over faces coef_f (u_a - u_nb): the
// "plus" face of a node carries fx[a] / fy[a]; its "minus" face is the plus
// face of the minus neighbour.  Faces past a Neumann end do not exist.
void five_point_row(const Geom& g, const std::vector<double>& fx, const std::vector<double>& fy, int a,
                    Row& r) {
  const int i = a / g.ny, j = a % g.ny;
  r.n = 0;
  r.add(a, 0.0);
  auto face = [&](int nb, double c) {
    r.add(a, c);
    r.add(nb, -c);
  };
  if (g.actx) {
    if (g.perx || i < g.nx - 1) face(((i + 1) % g.nx) * g.ny + j, fx[(size_t)a]);
    if (g.perx || i > 0) {
      const int im = (i + g.nx - 1) % g.nx;
      face(im * g.ny + j, fx[(size_t)im * g.ny + j]);
    }
  }
  if (g.pery || j < g.ny - 1) face(i * g.ny + (j + 1) % g.ny, fy[(size_t)a]);
  if (g.pery || j > 0) {
    const int jm = (j + g.ny - 1) % g.ny;
    face(i * g.ny + jm, fy[(size_t)i * g.ny + jm]);
  }
}

// In-place banded Cholesky of an SPD matrix in lower column storage
// A[j (w+1) + (i - j)], 0 <= i - j <= w.  Returns false on a non-positive or
// non-finite pivot.
bool band_cholesky(std::vector<double>& A, int S, int w) {
  const size_t ld = (size_t)w + 1;
  for (int j = 0; j < S; ++j) {
    double* cj = &A[(size_t)j * ld];
    const double d = cj[0];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double ljj = std::sqrt(d), inv = 1.0 / ljj;
    cj[0] = ljj;
    const int m = std::min(w, S - 1 - j);
    for (int e = 1; e <= m; ++e) cj[e] *= inv;
    for (int e1 = 1; e1 <= m; ++e1) {
      const double lk = cj[e1];
      if (lk == 0.0) continue;
      double* ck = &A[(size_t)(j + e1) * ld];
      for (int e2 = e1; e2 <= m; ++e2) ck[e2 - e1] -= cj[e2] * lk;
    }
  }
  return true;
}

template <typename T>
T* upload_vec(const std::vector<T>& h) {
  T* d = nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(T)) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  return d;
}

// padded row length: a multiple of 16 bytes so every row starts 16-byte aligned
int band_row_words(int w, size_t elt) {
  const int per16 = (int)(16 / elt);
  return (w + 1 + per16 - 1) / per16 * per16;
}

// Launch shape of the substitutions.  G, the block of steps: the largest power
// of two <= 32 with 2G <= w (the pipelined schedule below needs the next
// block inside the band) whose stage (G factor rows, plus the G x G inverse of
// the block's triangle when G >= 4) fits in kBandStageBytes.  The half-width
// w is at least 2 (padded with zero coefficients), so G = 1 always fits.
struct BandShape {
  int wp, G, inv, stage, threads;
  size_t smem;
};

template <typename T>
BandShape band_shape(int w) {
  BandShape b;
  b.wp = band_row_words(w, sizeof(T));
  auto stage = [&](int G) { return G * b.wp + (G >= 4 ? G * G : 0); };
  b.G = 1;
  while (b.G < 32 && 4 * b.G <= w && (size_t)stage(b.G * 2) * sizeof(T) <= (size_t)kBandStageBytes) b.G *= 2;
  b.inv = b.G >= 4;
  b.stage = stage(b.G);
  // warp 0 solves the blocks; warps 1.. take the w - G far entries
  b.threads = std::min(512, std::max(64, 32 + (w - b.G + 31) / 32 * 32));
  const size_t rg = ((size_t)kBandRing * b.G + 3) / 4 * 4;
  b.smem = sizeof(T) * ((size_t)kBandRing * b.stage + rg + 64 + (size_t)w + b.G);
  return b;
}

// Factor rows in step order (the order the substitutions consume them),
// padded to a whole number of blocks: step t of the forward solve L y = b is
// band row t, with row (1/L_tt, L_{t+1,t}, ..., L_{t+w,t}); step t of the
// backward solve L^T x = y is band row j = S-1-t, with row (1/L_jj, L_{j,j-1},
// ..., L_{j,j-w}).  Entry d of a row couples step t to step t + d.  Padding
// steps (t >= S) carry 1/L = 1 and no coupling.  For G >= 4 every block also
// stores the transposed inverse of its G x G step-space triangle.
template <typename T>
int build_factors(const Geom& g, const std::vector<Row>& chat, const std::vector<Row>& lhat,
                  const std::vector<int>& ipos, const double* lamt, int w, PrecTables* t,
                  std::string* err) {
  const int S = g.S, nt = g.nt;
  const BandShape bs = band_shape<T>(w);
  const int G = bs.G, wp = bs.wp;
  const int Sp = (S + G - 1) / G * G, nblk = Sp / G;
  const size_t per = (size_t)Sp * wp;
  const size_t perD = bs.inv ? (size_t)nblk * G * G : 0;
  std::vector<T> Fc(per * nt, T(0)), Fr(per * nt, T(0));
  std::vector<T> Dc(perD * nt, T(0)), Dr(perD * nt, T(0));
  std::vector<int> bad((size_t)nt, 0);
  auto work = [&](int k0, int k1) {
    std::vector<double> A((size_t)S * (w + 1));
    std::vector<double> Tm((size_t)G * G), Ti((size_t)G * G);
    for (int k = k0; k < k1; ++k) {
      std::fill(A.begin(), A.end(), 0.0);
      for (int a = 0; a < S; ++a) {
        const int pa = ipos[(size_t)a];
        auto put = [&](const Row& r, double scale) {
          for (int q = 0; q < r.n; ++q) {
            const int pc = ipos[(size_t)r.col[q]];
            if (pc < pa) continue;  // lower triangle in column storage: (row pc, col pa), pc >= pa
            A[(size_t)pa * (w + 1) + (pc - pa)] += scale * r.val[q];
          }
        };
        put(chat[(size_t)a], 1.0);
        put(lhat[(size_t)a], lamt[k]);
      }
      if (!band_cholesky(A, S, w)) {
        bad[(size_t)k] = 1;
        continue;
      }
      // coupling of step tt to step tt + d in direction dir, 0 outside the matrix
      auto coef = [&](int dir, int tt, int d) -> double {
        if (tt >= S || tt + d >= S) return 0.0;
        const int col = dir == 0 ? tt : S - 1 - tt - d;  // column of L in band storage
        return A[(size_t)col * (w + 1) + d];
      };
      auto diag = [&](int dir, int tt) -> double {
        if (tt >= S) return 1.0;
        return A[(size_t)(dir == 0 ? tt : S - 1 - tt) * (w + 1)];
      };
      for (int dir = 0; dir < 2; ++dir) {
        T* F = (dir == 0 ? Fc.data() : Fr.data()) + per * k;
        for (int tt = 0; tt < Sp; ++tt) {
          F[(size_t)tt * wp] = (T)(1.0 / diag(dir, tt));
          for (int d = 1; d <= w; ++d) F[(size_t)tt * wp + d] = (T)coef(dir, tt, d);
        }
        if (!bs.inv) continue;
        // Step-space triangle of each block (steps t0 .. t0+G-1), inverted by
        // forward substitution in FP64, stored transposed.
        T* D = (dir == 0 ? Dc.data() : Dr.data()) + perD * k;
        for (int blk = 0; blk < nblk; ++blk) {
          const int t0 = blk * G;
          std::fill(Tm.begin(), Tm.end(), 0.0);
          for (int a = 0; a < G; ++a) {
            Tm[(size_t)a * G + a] = diag(dir, t0 + a);
            for (int b = 0; b < a; ++b)
              if (a - b <= w) Tm[(size_t)a * G + b] = coef(dir, t0 + b, a - b);
          }
          for (int c = 0; c < G; ++c)
            for (int a = 0; a < G; ++a) {
              double v = (a == c) ? 1.0 : 0.0;
              for (int b = c; b < a; ++b) v -= Tm[(size_t)a * G + b] * Ti[(size_t)b * G + c];
              Ti[(size_t)a * G + c] = (a >= c) ? v / Tm[(size_t)a * G + a] : 0.0;
            }
          T* Db = D + (size_t)blk * G * G;
          for (int a = 0; a < G; ++a)
            for (int b = 0; b < G; ++b) Db[(size_t)b * G + a] = (T)Ti[(size_t)a * G + b];
        }
      }
    }
  };
  const int nth = std::max(1, std::min(nt, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int q = 0; q < nth; ++q) pool.emplace_back(work, q * nt / nth, (q + 1) * nt / nth);
  for (auto& th : pool) th.join();
  for (int k = 0; k < nt; ++k)
    if (bad[(size_t)k]) {
      *err = "viscosity field: a per-frequency system is not positive definite";
      return MFG_ERR_INVALID_ARG;
    }
  T* dc = upload_vec(Fc);
  T* dr = upload_vec(Fr);
  T* ic = bs.inv ? upload_vec(Dc) : nullptr;
  T* ir = bs.inv ? upload_vec(Dr) : nullptr;
  if constexpr (sizeof(T) == 8) {
    t->bandc64 = dc;
    t->bandr64 = dr;
    t->bandic64 = ic;
    t->bandir64 = ir;
  } else {
    t->bandc32 = dc;
    t->bandr32 = dr;
    t->bandic32 = ic;
    t->bandir32 = ir;
  }
  if (!dc || !dr || (bs.inv && (!ic || !ir))) {
    *err = "cudaMalloc failed for the banded factors";
    return MFG_ERR_CUDA;  // the caller frees what was uploaded
  }
  return MFG_OK;
}

}  // namespace

int build_band_tables(const mfg_problem& p, const Geom& g, const double* lamt, PrecTables* t,
                      std::string* err) {
  const int S = g.S;
  // node viscosities on the internal (nx, ny) grid: the caller's [Nx][Ny]
  // array, which for d = 1 is the N values along the internal y axis
  const double* nu = p.nu_field;
  std::vector<double> fx((size_t)S, 0.0), fy((size_t)S, 0.0), ux((size_t)S, 0.0), uy((size_t)S, 0.0);
  for (int i = 0; i < g.nx; ++i)
    for (int j = 0; j < g.ny; ++j) {
      const size_t a = (size_t)i * g.ny + j;
      if (g.actx && (g.perx || i < g.nx - 1)) {
        const size_t b = (size_t)((i + 1) % g.nx) * g.ny + j;
        fx[a] = 0.5 * (nu[a] + nu[b]) * g.ax;
        ux[a] = g.ax;
      }
      if (g.pery || j < g.ny - 1) {
        const size_t b = (size_t)i * g.ny + (j + 1) % g.ny;
        fy[a] = 0.5 * (nu[a] + nu[b]) * g.ay;
        uy[a] = g.ay;
      }
    }
  // band order
  const std::vector<int> rx = axis_rank(g.nx, g.perx), ry = axis_rank(g.ny, g.pery);
  std::vector<int> ipos((size_t)S);
  for (int i = 0; i < g.nx; ++i)
    for (int j = 0; j < g.ny; ++j) ipos[(size_t)i * g.ny + j] = rx[(size_t)i] * g.ny + ry[(size_t)j];
  // rows of K_nu and K, then C_hat = K_nu^2 + 2K and L_hat = (K_nu + I/dt)/dt
  std::vector<Row> kv((size_t)S), chat((size_t)S), lhat((size_t)S);
  for (int a = 0; a < S; ++a) five_point_row(g, fx, fy, a, kv[(size_t)a]);
  const double idt = g.idt;
  int w = 0;
  for (int a = 0; a < S; ++a) {
    Row k1;
    five_point_row(g, ux, uy, a, k1);
    Row& c = chat[(size_t)a];
    const Row& ra = kv[(size_t)a];
    for (int q = 0; q < ra.n; ++q) {
      const Row& rb = kv[(size_t)ra.col[q]];
      for (int u = 0; u < rb.n; ++u) c.add(rb.col[u], ra.val[q] * rb.val[u]);
    }
    for (int q = 0; q < k1.n; ++q) c.add(k1.col[q], 2.0 * k1.val[q]);
    Row& l = lhat[(size_t)a];
    for (int q = 0; q < ra.n; ++q) l.add(ra.col[q], ra.val[q] * idt);
    l.add(a, idt * idt);
    for (int q = 0; q < c.n; ++q) w = std::max(w, std::abs(ipos[(size_t)c.col[q]] - ipos[(size_t)a]));
  }
  w = std::max(w, 2);  // the pipelined substitutions need 2G <= w with G >= 1
  const size_t elt = p.precision == MFG_FP64 ? 8 : 4;
  const double bytes = 2.0 * g.nt * (double)S * band_row_words(w, elt) * elt;
  if (w > kBandMaxW || bytes > kBandMaxBytes) {
    *err = "viscosity field: banded factors too large (half-bandwidth " + std::to_string(w) +
           ", " + std::to_string(bytes / 1073741824.0) + " GiB)";
    return MFG_ERR_UNSUPPORTED;
  }
  t->band_w = w;
  t->kfx = upload_vec(fx);
  t->kfy = upload_vec(fy);
  t->band_perm = upload_vec(ipos);
  if (!t->kfx || !t->kfy || !t->band_perm) {
    *err = "cudaMalloc failed for the viscosity tables";
    return MFG_ERR_CUDA;
  }
  if (p.precision == MFG_FP64) return build_factors<double>(g, chat, lhat, ipos, lamt, w, t, err);
  return build_factors<float>(g, chat, lhat, ipos, lamt, w, t, err);
}

// ---------------------------------------------------------------- device --
namespace {

template <int B>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// One bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16) that completes on the mbarrier at `mbar`.
__device__ __forceinline__ void bulk_load(void* smem, const void* gmem, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(smem)),
      "l"(gmem), "r"(bytes), "r"(mbar)
      : "memory");
}
constexpr uint32_t kBandPolls = 1u << 22;  // mbarrier polls before a wait gives up
// Waits for phase `parity` of the mbarrier, giving up after `polls` polls.
__device__ __forceinline__ bool band_wait(uint32_t mbar, uint32_t parity, uint32_t polls) {
  for (uint32_t it = 0; it < polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Time transform of every spatial point: out[k][.] = sum_j V[k][j] in[j][.]
// (V symmetric and orthonormal, so the same product is forward and inverse).
// TO_BAND: outputs go to band positions ipos[s]; FROM_BAND: inputs are read
// from them.  A block holds a strip of 32 points x N_t levels in shared memory;
// lanes own points, warps own output levels.
template <typename TI, typename TO, typename T, bool FROM_BAND, bool TO_BAND>
__global__ void __launch_bounds__(256) k_time_xf(const TI* __restrict__ in, TO* __restrict__ out,
                                                 const T* __restrict__ V, const int* __restrict__ ipos,
                                                 int nt, int S, const DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* strip = reinterpret_cast<T*>(smraw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + lane;
  const bool ok = s < S;
  const int ps = ok ? ipos[s] : 0;
  const long long src = FROM_BAND ? ps : s, dst = TO_BAND ? ps : s;
  for (int j = wid; j < nt; j += 8) strip[j * 32 + lane] = ok ? (T)in[(long long)j * S + src] : T(0);
  __syncthreads();
  if (!ok) return;
  for (int k = wid; k < nt; k += 8) {
    const T* vr = V + (size_t)k * nt;
    T acc = T(0);
    for (int j = 0; j < nt; ++j) acc = fma(vr[j], strip[j * 32 + lane], acc);
    out[(long long)k * S + dst] = (TO)acc;
  }
}

// xr[0..G) = xs[0..G) with 16-byte shared loads (xs is 16-byte aligned)
template <typename T, int G>
__device__ __forceinline__ void load_block(const T* xs, T (&xr)[G]) {
  constexpr int V = 16 / (int)sizeof(T);
  if constexpr (G % V == 0 && sizeof(T) == 4) {
#pragma unroll
    for (int b = 0; b < G; b += 4) {
      const float4 q = *reinterpret_cast<const float4*>(xs + b);
      xr[b] = q.x; xr[b + 1] = q.y; xr[b + 2] = q.z; xr[b + 3] = q.w;
    }
  } else if constexpr (G % V == 0 && sizeof(T) == 8) {
#pragma unroll
    for (int b = 0; b < G; b += 2) {
      const double2 q = *reinterpret_cast<const double2*>(xs + b);
      xr[b] = q.x; xr[b + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int b = 0; b < G; ++b) xr[b] = xs[b];
  }
}

// One banded substitution per frequency (blockIdx.x = k).  Both directions are
// the same lower-triangular banded solve in step order t = 0..S'-1 (S' = S
// rounded up to whole blocks; padding steps have a unit diagonal, no coupling
// and a zero right-hand side): row t of F holds 1/L_tt and the coefficients
// coupling step t to steps t+1 .. t+w (forward: band row t of L; backward:
// band row S-1-t of L^T).  Steps go in blocks of G (a power of two <= 32,
// 2G <= w) with a one-block lag between the two kinds of work:
//   warp 0 solves block st: its right-hand side is the window entry less
//     `carry`, the contribution of block st-1 that warp 0 computed itself; the
//     G x G triangle is one product with its inverse for G >= 4 (formed on the
//     host in FP64 and streamed with the rows; lane a sums G terms, no
//     dependency chain), else a shuffle chain; then it forms block st's
//     contribution to block st+1 (distances G+l-b <= 2G-1 <= w) in `carry`;
//   warps 1.. meanwhile subtract block st-1's contribution from entries
//     t0+G .. t0+w-1 (distance 2G+e-b, zero past w) and copy the right-hand
//     side of entries t0+w .. t0+w+G-1 into the window.
// One barrier per block.  The window keeps entry t at slot t mod (w+G): during
// block st it holds entries t0 .. t0+w+G-1, the new entries taking the slots
// of block st-1, which nothing reads any more.  The solutions of blocks st and
// st-1 sit in two halves of xs.  Factor rows, block inverses and right-hand
// sides of a block arrive through a ring of kBandRing shared-memory stages
// kBandRing-2 blocks ahead (stage st-1 is still read during block st): the
// rows and the inverse of a block are contiguous in global memory, so one
// thread issues them as bulk copies that complete on the stage's mbarrier,
// which warp 0 waits on before the block's barrier; warp 1 fetches the G
// right-hand-side values with 4- or 8-byte cp.async copies.  Every wait is
// bounded: a stage that never arrives marks this frequency's output NaN,
// records MFG_ERR_TIMEOUT and ends the kernel.
template <typename T, bool BWD, int G>
__global__ void __launch_bounds__(512) k_band_pass(const T* __restrict__ rhs, T* __restrict__ sol,
                                                    const T* __restrict__ F, const T* __restrict__ Dinv,
                                                    int S, int w, int wp, DevScalars* sc) {
  constexpr bool INV = G >= 4;                        // blocks carry their triangle's inverse
  constexpr int RG = (kBandRing * G + 3) / 4 * 4;     // right-hand-side stages, 16-byte multiple
  if (sc != nullptr && sc->cg_done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int stage = G * wp + (INV ? G * G : 0);
  T* ring = reinterpret_cast<T*>(smraw);              // kBandRing x (G rows of wp [+ G x G inverse])
  T* refill = ring + (size_t)kBandRing * stage;       // kBandRing x G
  T* xs = refill + RG;                                // 2 x 32
  T* win = xs + 64;                                   // w + G
  const int k = blockIdx.x, tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int wt = tid - 32, wn = nth - 32;             // rank among warps 1..
  const int W2 = w + G;
  const int Sp = (S + G - 1) / G * G, nblk = Sp / G;
  const T* Fk = F + (size_t)k * Sp * wp;
  const T* Dk = INV ? Dinv + (size_t)k * nblk * G * G : nullptr;
  const T* bk = rhs + (size_t)k * S;
  T* xk = sol + (size_t)k * S;
  auto band = [&](int t) { return BWD ? S - 1 - t : t; };
  __shared__ __align__(8) unsigned long long mbar[kBandRing];
  const uint32_t rowbytes = (uint32_t)((size_t)G * wp * sizeof(T));
  const uint32_t invbytes = INV ? (uint32_t)((size_t)G * G * sizeof(T)) : 0u;
  auto issue = [&](int st) {
    if (warp != 1) return;
    if (st < nblk) {
      const int t0 = st * G;
      T* dst = ring + (size_t)(st % kBandRing) * stage;
      if (lane == 0) {
        const uint32_t mb = smem_addr(&mbar[st % kBandRing]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(rowbytes + invbytes)
                     : "memory");
        bulk_load(dst, Fk + (size_t)t0 * wp, rowbytes, mb);
        if constexpr (INV) bulk_load(dst + (size_t)G * wp, Dk + (size_t)st * G * G, invbytes, mb);
      }
      if (lane < G) {
        const int r = t0 + w + lane;
        T* rf = refill + (st % kBandRing) * G + lane;
        if (r < S)
          cp_async_small<sizeof(T)>(rf, bk + band(r));
        else
          *rf = T(0);  // padding step
      }
    }
    cp_async_commit();
  };
  if (tid == 0) {
    for (int i = 0; i < kBandRing; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  for (int e = tid; e < w && e < Sp; e += nth) win[e] = e < S ? bk[band(e)] : T(0);
  for (int st = 0; st < kBandRing - 2; ++st) issue(st);
  // slot of entry t0 + x is s0 + x, less W2 past the end (x < W2): no divisions
  int s0 = 0;
  auto slot = [&](int x) { const int q = s0 + x; return q >= W2 ? q - W2 : q; };
  T carry = T(0);
  const int ml = lane < G ? lane : 0;
  int failed = 0;
  for (int st = 0; st < nblk; ++st) {
    bool ok = true;
    if (warp == 0) ok = band_wait(smem_addr(&mbar[st % kBandRing]), (uint32_t)(st / kBandRing) & 1u, kBandPolls);
    if (warp == 1) cp_async_wait<kBandRing - 3>();
    if (__syncthreads_or(ok ? 0 : 1)) {
      failed = st + 1;
      break;
    }
    issue(st + kBandRing - 2);
    const int t0 = st * G;
    const T* cur = ring + (size_t)(st % kBandRing) * stage;
    if (warp == 0) {
      T acc = lane < G ? win[slot(lane)] - carry : T(0);
      T x = T(0);
      if constexpr (INV) {
        // x = T^{-1} acc with the block's inverse (transposed in the stage)
        const T* Di = cur + (size_t)G * wp;
        T xa[4] = {T(0), T(0), T(0), T(0)};  // four independent FMA chains
#pragma unroll
        for (int b = 0; b < G; ++b) xa[b & 3] = fma(Di[b * G + ml], __shfl_sync(0xffffffffu, acc, b), xa[b & 3]);
        x = (xa[0] + xa[1]) + (xa[2] + xa[3]);
      } else {
        const T inv = cur[(size_t)ml * wp];
#pragma unroll
        for (int b = 0; b < G; ++b) {
          const T xb = __shfl_sync(0xffffffffu, acc * inv, b);
          if (lane == b) x = xb;
          if (lane > b && lane < G) acc = fma(-cur[(size_t)b * wp + (lane - b)], xb, acc);
        }
      }
      T* xc = xs + (st & 1) * 32;
      if (lane < G) {
        xc[lane] = x;
        if (t0 + lane < S) xk[band(t0 + lane)] = x;
      }
      __syncwarp();
      T xr[G];
      load_block<T, G>(xc, xr);
      T cs[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int b = 0; b < G; ++b) cs[b & 3] = fma(cur[(size_t)b * wp + (G + ml - b)], xr[b], cs[b & 3]);
      carry = (cs[0] + cs[1]) + (cs[2] + cs[3]);
    } else {
      if (st > 0) {
        const T* prv = ring + (size_t)((st + kBandRing - 1) % kBandRing) * stage;
        T xr[G];
        load_block<T, G>(xs + ((st - 1) & 1) * 32, xr);
        const int ne = min(w - G, Sp - t0 - G);
        for (int e = wt; e < ne; e += wn) {
          T acc[4] = {T(0), T(0), T(0), T(0)};  // four independent FMA chains
          if (2 * G + e <= w) {                   // every row of block st-1 reaches entry t0+G+e
#pragma unroll
            for (int b = 0; b < G; ++b) acc[b & 3] = fma(prv[(size_t)b * wp + (2 * G + e - b)], xr[b], acc[b & 3]);
          } else {
#pragma unroll
            for (int b = 0; b < G; ++b) {
              const int d = 2 * G + e - b;
              const T v = prv[(size_t)b * wp + (d <= w ? d : 0)];  // in-bounds address either way
              if (d <= w) acc[b & 3] = fma(v, xr[b], acc[b & 3]);
            }
          }
          win[slot(G + e)] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
      }
      if (wt < G && t0 + w + wt < Sp) win[slot(w + wt)] = refill[(st % kBandRing) * G + wt];
    }
    s0 = slot(G);
  }
  cp_async_wait<0>();
  if (failed) {
    // stage failed-1 never arrived: let the stages still in flight land
    // (bounded) before the shared memory goes away, and mark the output
    const int st = failed - 1;
    if (tid == 0)
      for (int j = st; j < min(nblk, st + kBandRing - 2); ++j)
        band_wait(smem_addr(&mbar[j % kBandRing]), (uint32_t)(j / kBandRing) & 1u, kBandPolls);
    for (int t = tid; t < S; t += nth) xk[t] = (T)__int_as_float(0x7fc00000);
    if (tid == 0 && sc != nullptr) {
      sc->status = MFG_ERR_TIMEOUT;
      sc->cg_done = 1;
    }
    __syncthreads();
  }
}

template <typename T, bool BWD>
void launch_band_pass(const BandShape& b, int nt, const T* in, T* out, const T* F, const T* Dinv, int S,
                      int w, const DevScalars* sc, cudaStream_t s) {
  DevScalars* scw = const_cast<DevScalars*>(sc);  // written only when a bounded wait runs out
  switch (b.G) {
#define MFG_BAND_G(GG) \
  case GG: k_band_pass<T, BWD, GG><<<nt, b.threads, b.smem, s>>>(in, out, F, Dinv, S, w, b.wp, scw); break;
    MFG_BAND_G(32) MFG_BAND_G(16) MFG_BAND_G(8) MFG_BAND_G(4) MFG_BAND_G(2) MFG_BAND_G(1)
#undef MFG_BAND_G
    default: break;
  }
}

template <typename T>
void precond_band_typed(const Geom& g, const PrecTables& t, const T* V, const T* Lc, const T* Lr,
                        const T* Ic, const T* Ir, const double* r, double* z, T* w0, T* w1,
                        const DevScalars* sc, cudaStream_t s) {
  const int S = g.S, nt = g.nt, w = t.band_w;
  const size_t tsm = sizeof(T) * (size_t)nt * 32;
  const int tb = (S + 31) / 32;
  k_time_xf<double, T, T, false, true><<<tb, 256, tsm, s>>>(r, w0, V, t.band_perm, nt, S, sc);
  const BandShape b = band_shape<T>(w);
  launch_band_pass<T, false>(b, nt, w0, w1, Lc, Ic, S, w, sc, s);
  launch_band_pass<T, true>(b, nt, w1, w0, Lr, Ir, S, w, sc, s);
  k_time_xf<T, double, T, true, false><<<tb, 256, tsm, s>>>(w0, z, V, t.band_perm, nt, S, sc);
}

template <typename T>
int band_attrs(int smem) {
  int bad = 0;
#define MFG_BAND_ATTR(GG)                                                                                \
  bad |= cudaFuncSetAttribute(k_band_pass<T, false, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != \
         cudaSuccess;                                                                                    \
  bad |= cudaFuncSetAttribute(k_band_pass<T, true, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess;
  MFG_BAND_ATTR(32) MFG_BAND_ATTR(16) MFG_BAND_ATTR(8) MFG_BAND_ATTR(4) MFG_BAND_ATTR(2) MFG_BAND_ATTR(1)
#undef MFG_BAND_ATTR
  return bad;
}

}  // namespace

// Largest dynamic shared memory the band kernels ask for (half-bandwidth up
// to kBandMaxW); called once per device before any launch or capture.
int band_configure() {
  int bad = 0;
  size_t m64 = 0, m32 = 0;
  for (int w = 1; w <= kBandMaxW; ++w) {
    m64 = std::max(m64, band_shape<double>(w).smem);
    m32 = std::max(m32, band_shape<float>(w).smem);
  }
  bad |= band_attrs<double>((int)m64);
  bad |= band_attrs<float>((int)m32);
  const int t64 = (int)(sizeof(double) * kMaxNt * 32), t32 = (int)(sizeof(float) * kMaxNt * 32);
  bad |= cudaFuncSetAttribute(k_time_xf<double, double, double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, t64) != cudaSuccess;
  bad |= cudaFuncSetAttribute(k_time_xf<double, double, double, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, t64) != cudaSuccess;
  bad |= cudaFuncSetAttribute(k_time_xf<double, float, float, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, t32) != cudaSuccess;
  bad |= cudaFuncSetAttribute(k_time_xf<float, double, float, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, t32) != cudaSuccess;
  return bad ? MFG_ERR_CUDA : MFG_OK;
}

void launch_precond_band(const Geom& g, const PrecTables& t, int precision, const double* r, double* z,
                         double* work64, float* work32, const DevScalars* sc, cudaStream_t s) {
  if (precision == MFG_FP64)
    precond_band_typed<double>(g, t, t.Vt64, t.bandc64, t.bandr64, t.bandic64, t.bandir64, r, z, work64,
                               work64 + g.n, sc, s);
  else
    precond_band_typed<float>(g, t, t.Vt32, t.bandc32, t.bandr32, t.bandic32, t.bandir32, r, z, work32,
                              work32 + g.n, sc, s);
}

}  // namespace mfg
