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
// walks its S points in blocks of up to 32 steps.  Two warps solve a block
// (its inverted triangle and its map to the next block, both formed on the
// host), the other warps apply the previous block to the later partial sums
// (a circular window in shared memory), one block behind; each block's
// coefficients are one contiguous stage that a bulk copy brings into a ring
// of shared-memory stages a few blocks ahead, so the loads never wait on the
// dependency chain.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "mfg_internal.cuh"

namespace mfg {

namespace {

constexpr int kBandRing = 5;           // shared-memory stages of the substitutions
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

// Launch shape of the substitutions.  G, the block of steps: the largest power
// of two <= 32 with 2G <= w (the pipelined schedule below needs the next
// block inside the band) whose stage fits in kBandStageBytes.  A block's stage
// holds G (w + G) values, rounded up to 16 bytes: the G x G inverse of the
// block's triangle, the G x G map from the block's right-hand side to its
// contribution to the next block, and the coefficients of the w - G entries
// after that.  The half-width w is at least 2 (padded with zero
// coefficients), so G = 1 always fits.
struct BandShape {
  int G, stage, threads;
  size_t smem;
};

template <typename T>
BandShape band_shape(int w) {
  constexpr int V = 16 / (int)sizeof(T);
  BandShape b;
  auto stage = [&](int G) { return (G * (w + G) + V - 1) / V * V; };
  b.G = 1;
  while (b.G < 32 && 4 * b.G <= w && (size_t)stage(b.G * 2) * sizeof(T) <= (size_t)kBandStageBytes) b.G *= 2;
  b.stage = stage(b.G);
  // warps 0 and 1 solve the blocks, warp 2 moves the data, warps 3.. take
  // the w - G far entries
  b.threads = std::min(512, 96 + (w - b.G + 31) / 32 * 32);
  const size_t rg = ((size_t)kBandRing * b.G + 3) / 4 * 4;
  b.smem = sizeof(T) * ((size_t)kBandRing * b.stage + rg + 192 + (size_t)w + b.G);
  return b;
}

// Position of entry c of row r in a stage section of G-wide rows.  When a row
// is whole 16-byte chunks of V values (G a multiple of V), chunk q of row r
// sits at chunk q ^ (r mod G/V): eight consecutive rows read at one chunk
// index then fall in distinct banks.
inline int band_pos(int r, int c, int G, int V) {
  if (G % V != 0) return r * G + c;
  const int nq = G / V;
  return r * G + (((c / V) ^ (r & (nq - 1))) * V) + c % V;
}

// The substitution stages, in step order and padded to a whole number of
// blocks.  Step t of the forward solve L y = b is band row t; step t of the
// backward solve L^T x = y is band row S-1-t; coef(t, d) couples step t to
// step t + d (L_{t+d,t} forward, L_{j,j-d} with j = S-1-t backward).  Padding
// steps (t >= S) have a unit diagonal and no coupling.  For the block of steps
// t0 .. t0+G-1 with step-space triangle T_blk (computed in FP64):
//   rows l of section 0: row l of T_blk^{-1}           (x = T_blk^{-1} acc)
//   rows l of section 1: row l of N T_blk^{-1}, with N[l][a] = coef(t0+a,
//     G+l-a): the block's contribution to step t0+G+l, straight from acc
//   rows e of section 2, e < w-G: coef(t0+b, 2G+e-b) at entry b, zero past
//     the band: the block's contribution to step t0+2G+e.
template <typename T>
int build_factors(const Geom& g, const std::vector<Row>& chat, const std::vector<Row>& lhat,
                  const std::vector<int>& ipos, const double* lamt, int w, PrecTables* t,
                  std::string* err) {
  const int S = g.S, nt = g.nt;
  constexpr int V = 16 / (int)sizeof(T);
  const BandShape bs = band_shape<T>(w);
  const int G = bs.G, stg = bs.stage;
  const int Sp = (S + G - 1) / G * G, nblk = Sp / G;
  const size_t per = (size_t)nblk * stg;
  std::vector<T> Fc(per * nt, T(0)), Fr(per * nt, T(0));
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
      for (int dir = 0; dir < 2; ++dir) {
        // coupling of step tt to step tt + d (d <= w), 0 outside the matrix
        auto coef = [&](int tt, int d) -> double {
          if (tt >= S || tt + d >= S) return 0.0;
          const int col = dir == 0 ? tt : S - 1 - tt - d;  // column of L in band storage
          return A[(size_t)col * (w + 1) + d];
        };
        auto diag = [&](int tt) -> double {
          if (tt >= S) return 1.0;
          return A[(size_t)(dir == 0 ? tt : S - 1 - tt) * (w + 1)];
        };
        T* F = (dir == 0 ? Fc.data() : Fr.data()) + per * k;
        for (int blk = 0; blk < nblk; ++blk) {
          const int t0 = blk * G;
          T* B = F + (size_t)blk * stg;
          std::fill(Tm.begin(), Tm.end(), 0.0);
          for (int a = 0; a < G; ++a) {
            Tm[(size_t)a * G + a] = diag(t0 + a);
            for (int c = 0; c < a; ++c) Tm[(size_t)a * G + c] = coef(t0 + c, a - c);  // a - c < G <= w
          }
          // inverse of the lower triangle by forward substitution, column by column
          for (int c = 0; c < G; ++c)
            for (int a = 0; a < G; ++a) {
              double v = (a == c) ? 1.0 : 0.0;
              for (int m = c; m < a; ++m) v -= Tm[(size_t)a * G + m] * Ti[(size_t)m * G + c];
              Ti[(size_t)a * G + c] = (a >= c) ? v / Tm[(size_t)a * G + a] : 0.0;
            }
          for (int l = 0; l < G; ++l)
            for (int c = 0; c < G; ++c) {
              B[band_pos(l, c, G, V)] = (T)Ti[(size_t)l * G + c];
              double m = 0.0;  // (N T^{-1})[l][c], T^{-1} lower triangular
              for (int a = c; a < G; ++a) m += coef(t0 + a, G + l - a) * Ti[(size_t)a * G + c];
              B[(size_t)G * G + band_pos(l, c, G, V)] = (T)m;
            }
          for (int e = 0; e < w - G; ++e)
            for (int c = 0; c < G; ++c) {
              const int d = 2 * G + e - c;
              B[(size_t)2 * G * G + band_pos(e, c, G, V)] = d <= w ? (T)coef(t0 + c, d) : T(0);
            }
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
  if constexpr (sizeof(T) == 8) {
    t->bandc64 = dc;
    t->bandr64 = dr;
  } else {
    t->bandc32 = dc;
    t->bandr32 = dr;
  }
  if (!dc || !dr) {
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
  const double bytes = 2.0 * g.nt * ((double)S + 32) * (w + 32) * elt;  // stages: G (w + G) per G steps
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
// Poll limit under the fault-injection hook (no copy issued, nothing ever
// arrives): short, so the test of the timeout path costs milliseconds.
constexpr uint32_t kBandPollsInjected = 1u << 12;
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

// Dot product of row r of a stage section (G-wide rows, layout band_pos)
// with xr: 16-byte loads when rows are whole chunks, four FMA chains.
template <typename T, int G>
__device__ __forceinline__ T row_dot(const T* sec, int r, const T (&xr)[G]) {
  constexpr int V = 16 / (int)sizeof(T);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  const T* row = sec + r * G;
  if constexpr (G % V == 0) {
    constexpr int NQ = G / V;
    const int sw = r & (NQ - 1);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const T* p = row + ((q ^ sw) * V);
      if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        acc[0] = fma(v.x, xr[4 * q], acc[0]);
        acc[1] = fma(v.y, xr[4 * q + 1], acc[1]);
        acc[2] = fma(v.z, xr[4 * q + 2], acc[2]);
        acc[3] = fma(v.w, xr[4 * q + 3], acc[3]);
      } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        acc[(2 * q) & 3] = fma(v.x, xr[2 * q], acc[(2 * q) & 3]);
        acc[(2 * q + 1) & 3] = fma(v.y, xr[2 * q + 1], acc[(2 * q + 1) & 3]);
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < G; ++c) acc[c & 3] = fma(row[c], xr[c], acc[c & 3]);
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// One banded substitution per frequency (blockIdx.x = k).  Both directions are
// the same lower-triangular banded solve in step order t = 0..S'-1 (S' = S
// rounded up to whole blocks of G steps; G a power of two <= 32 with
// 2G <= w), with a one-block lag between the kinds of work:
//   warps 0 and 1 solve block st.  Its right-hand side acc is the window
//     entries less `carry`, block st-1's contribution to them, which warp 1
//     formed in the previous block.  Both warps read all of acc; lane l of
//     warp 0 forms x_l = (T^{-1} acc)_l and lane l of warp 1 the next carry
//     (N T^{-1} acc)_l, each a G-term dot product with a row of the block's
//     stage (the host formed both matrices in FP64);
//   warp 2 issues the copies of block st+kBandRing-2 and moves the right-hand
//     side of entries t0+w .. t0+w+G-1 into the window;
//   warps 3.. subtract block st-1's contribution from entries t0+G .. t0+w-1
//     (thread e: one G-term dot product with row e of the far section, zeros
//     past the band).
// One barrier per block.  The window keeps entry t at slot t mod (w+G): during
// block st it holds entries t0 .. t0+w+G-1, the new entries taking the slots
// of block st-1, which nothing reads any more.  The solutions of blocks st and
// st-1 sit in two halves of xs.  Each block's stage is contiguous in global
// memory and arrives through a ring of kBandRing shared-memory stages
// kBandRing-2 blocks ahead (stage st-1 is still read during block st): one
// thread issues it as a bulk copy that completes on the stage's mbarrier,
// which warp 0 waits on before the block's barrier; warp 2 fetches the G
// right-hand-side values with 4- or 8-byte cp.async copies.  Every wait is
// bounded: a stage that never arrives marks this frequency's output NaN,
// records MFG_ERR_TIMEOUT and ends the kernel.
template <typename T, bool BWD, int G>
__global__ void __launch_bounds__(512, 1) k_band_pass(const T* __restrict__ rhs, T* __restrict__ sol,
                                                    const T* __restrict__ F, int S, int w, int stage,
                                                    DevScalars* sc) {
  constexpr int RG = (kBandRing * G + 3) / 4 * 4;     // right-hand-side stages, 16-byte multiple
  if (sc != nullptr && sc->cg_done) return;
  // Fault-injection hook (MFG_INJECT_BAND_NO_COPY): no stage copy and no
  // expected-bytes arrival are issued, so the bounded stage wait must run out.
  const bool no_copy = sc != nullptr && sc->inject == MFG_INJECT_BAND_NO_COPY;
  const uint32_t polls = no_copy ? kBandPollsInjected : kBandPolls;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* ring = reinterpret_cast<T*>(smraw);              // kBandRing stages
  T* refill = ring + (size_t)kBandRing * stage;       // kBandRing x G
  T* xs = refill + RG;                                // 2 x 32
  T* accb = xs + 64;                                  // 2 x 32: the block's right-hand side (warps 0, 1)
  T* cb = accb + 64;                                  // 2 x 32: carry of the current and previous block
  T* win = cb + 64;                                   // w + G
  const int k = blockIdx.x, tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int wt = tid - 96, wn = nth - 96;             // rank among warps 3..
  const int W2 = w + G;
  const int Sp = (S + G - 1) / G * G, nblk = Sp / G;
  const T* Fk = F + (size_t)k * nblk * stage;
  const T* bk = rhs + (size_t)k * S;
  T* xk = sol + (size_t)k * S;
  auto band = [&](int t) { return BWD ? S - 1 - t : t; };
  __shared__ __align__(8) unsigned long long mbar[kBandRing];
  const uint32_t sbytes = (uint32_t)((size_t)stage * sizeof(T));
  auto issue = [&](int st) {
    if (warp != 2) return;
    if (st < nblk) {
      const int t0 = st * G;
      if (lane == 0 && !no_copy) {
        const uint32_t mb = smem_addr(&mbar[st % kBandRing]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(sbytes) : "memory");
        bulk_load(ring + (size_t)(st % kBandRing) * stage, Fk + (size_t)st * stage, sbytes, mb);
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
  if (tid < 64) cb[tid] = T(0);
  __syncthreads();
  for (int e = tid; e < w && e < Sp; e += nth) win[e] = e < S ? bk[band(e)] : T(0);
  for (int st = 0; st < kBandRing - 2; ++st) issue(st);
  // slot of entry t0 + x is s0 + x, less W2 past the end (x < W2): no divisions
  int s0 = 0;
  auto slot = [&](int x) { const int q = s0 + x; return q >= W2 ? q - W2 : q; };
  const int ml = lane < G ? lane : 0;
  int failed = 0;
  for (int st = 0; st < nblk; ++st) {
    bool ok = true;
    if (warp == 0) ok = band_wait(smem_addr(&mbar[st % kBandRing]), (uint32_t)(st / kBandRing) & 1u, polls);
    if (warp == 2) cp_async_wait<kBandRing - 3>();
    if (__syncthreads_or(ok ? 0 : 1)) {
      failed = st + 1;
      break;
    }
    issue(st + kBandRing - 2);
    const int t0 = st * G;
    if (warp < 2) {
      const T* cur = ring + (size_t)(st % kBandRing) * stage;
      T* ab = accb + warp * 32;
      if (lane < G) ab[lane] = win[slot(lane)] - cb[((st + 1) & 1) * 32 + lane];
      __syncwarp();
      T ar[G];
      load_block<T, G>(ab, ar);
      if (warp == 0) {
        const T x = row_dot<T, G>(cur, ml, ar);
        if (lane < G) {
          xs[(st & 1) * 32 + lane] = x;
          if (t0 + lane < S) xk[band(t0 + lane)] = x;
        }
      } else {
        const T c = row_dot<T, G>(cur + G * G, ml, ar);
        if (lane < G) cb[(st & 1) * 32 + lane] = c;
      }
    } else if (warp == 2) {
      if (lane < G && t0 + w + lane < Sp) win[slot(w + lane)] = refill[(st % kBandRing) * G + lane];
    } else {
      if (st > 0) {
        const T* far = ring + (size_t)((st + kBandRing - 1) % kBandRing) * stage + 2 * G * G;
        T xr[G];
        load_block<T, G>(xs + ((st - 1) & 1) * 32, xr);
        const int ne = min(w - G, Sp - t0 - G);
        for (int e = wt; e < ne; e += wn) win[slot(G + e)] -= row_dot<T, G>(far, e, xr);
      }
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
        band_wait(smem_addr(&mbar[j % kBandRing]), (uint32_t)(j / kBandRing) & 1u, polls);
    for (int t = tid; t < S; t += nth) xk[t] = (T)__int_as_float(0x7fc00000);
    if (tid == 0 && sc != nullptr) {
      sc->status = MFG_ERR_TIMEOUT;
      sc->cg_done = 1;
    }
    __syncthreads();
  }
}

template <typename T, bool BWD>
void launch_band_pass(const BandShape& b, int nt, const T* in, T* out, const T* F, int S, int w,
                      const DevScalars* sc, cudaStream_t s) {
  DevScalars* scw = const_cast<DevScalars*>(sc);  // written only when a bounded wait runs out
  switch (b.G) {
#define MFG_BAND_G(GG) \
  case GG: k_band_pass<T, BWD, GG><<<nt, b.threads, b.smem, s>>>(in, out, F, S, w, b.stage, scw); break;
    MFG_BAND_G(32) MFG_BAND_G(16) MFG_BAND_G(8) MFG_BAND_G(4) MFG_BAND_G(2) MFG_BAND_G(1)
#undef MFG_BAND_G
    default: break;
  }
}

template <typename T>
void precond_band_typed(const Geom& g, const PrecTables& t, const T* V, const T* Fc, const T* Fr,
                        const double* r, double* z, T* w0, T* w1, const DevScalars* sc, cudaStream_t s) {
  const int S = g.S, nt = g.nt, w = t.band_w;
  const size_t tsm = sizeof(T) * (size_t)nt * 32;
  const int tb = (S + 31) / 32;
  k_time_xf<double, T, T, false, true><<<tb, 256, tsm, s>>>(r, w0, V, t.band_perm, nt, S, sc);
  const BandShape b = band_shape<T>(w);
  launch_band_pass<T, false>(b, nt, w0, w1, Fc, S, w, sc, s);
  launch_band_pass<T, true>(b, nt, w1, w0, Fr, S, w, sc, s);
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
    precond_band_typed<double>(g, t, t.Vt64, t.bandc64, t.bandr64, r, z, work64, work64 + g.n, sc, s);
  else
    precond_band_typed<float>(g, t, t.Vt32, t.bandc32, t.bandr32, r, z, work32, work32 + g.n, sc, s);
}

}  // namespace mfg
