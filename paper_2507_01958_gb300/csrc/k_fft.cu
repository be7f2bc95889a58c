// Spatial passes of the preconditioner by FFT, for axis lengths that are powers
// of two (Alg. 2: transform along y, then x, divide, invert).
//
// One block takes LB real lines of length N (rows of the contiguous y axis, or
// columns of the x axis), packs them pairwise into CL = LB/2 complex lines
// z = x_a + i x_b, runs a radix-4/2 Stockham FFT per complex line in shared
// memory (one warp per line, natural order in and out), and separates the
// pair with the Hermitian symmetry of real data:
//   X_a[k] = (Z[k] + conj Z[N-k]) / 2,  X_b[k] = (Z[k] - conj Z[N-k]) / (2i).
// Modes:
//   DHT  (periodic axis): H[k] = (Re X[k] - Im X[k]) / sqrt(N); its own inverse.
//   DCT2 (Neumann, forward): Makhoul's reordering v_n = x_{2n},
//        v_{N-1-n} = x_{2n+1}; C[k] = c_k Re(exp(-i pi k/(2N)) V[k]),
//        c_0 = sqrt(1/N), c_k = sqrt(2/N).
//   DCT3 (Neumann, inverse): V[k] = exp(i pi k/(2N)) (C[k]/c_k - i C[N-k]/c_{N-k}),
//        v = IFFT(V), x_{2n} = v_n, x_{2n+1} = v_{N-1-n}.
// The result equals the dense orthonormal transform of the plan's tables to
// round-off; the pass reads and writes each element once.
#include "mfg_internal.cuh"
#include "reduce.cuh"

namespace mfg {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T x, y;
};

enum { FFT_DHT = 0, FFT_DCT2 = 1, FFT_DCT3 = 2 };

// Lines of N >= 256 take radix-8 Stockham stages (N/8 >= 32 butterflies
// keep every lane of the warp busy), shorter lines radix-4 stages.
template <int N>
struct FftRadix {
  static constexpr bool R8 = N >= 256;
};

// Position of element k of a complex line in shared memory: k with its low
// four bits XORed by a mask taken from bits 4-7.  Stockham stages store with
// strides of R and R^2 elements, which without it send up to 8 lanes of a
// half-warp to one bank pair (8-byte elements).  Radix 8: mask 13 b4 ^ 9 b5 ^
// 14 b6 ^ 10 b7 (b_i = bit i of k), radix 4: 5 (b4 + 2 b5); each was chosen by
// searching over the stage, contiguous-load and separation access patterns,
// where it stays within 11 % (radix 8) of the minimum wavefront count.  Both
// permute within aligned groups of 16, so a line of N >= 8 stays in [0, N).
template <int N>
__device__ __forceinline__ int swz(int k) {
  if constexpr (FftRadix<N>::R8)
    return k ^ ((((k >> 4) & 1) * 13) ^ (((k >> 5) & 1) * 9) ^ (((k >> 6) & 1) * 14) ^ (((k >> 7) & 1) * 10));
  else
    return k ^ (((k >> 4) & 3) * 5);
}

template <typename T, int N>
struct FftShape {
  static constexpr int CL = 8;       // complex lines per block (one per warp)
  static constexpr int LB = 2 * CL;                                 // real lines per block
  static constexpr int NP = N + 1;  // padded line stride: staging across lines hits distinct banks
  static constexpr size_t smem = 2 * (size_t)CL * NP * sizeof(cx<T>) + (size_t)(N / 2 + N) * sizeof(cx<T>);
};

// Dot products fused into the last pass of a PCG preconditioner apply: while
// zp = P^{-1} r is stored, r.zp (and q.zp for the flexible variant) are
// accumulated and the last block forms beta exactly as k_dot_beta does.
struct DotFuse {
  const double* r;
  const double* q;
  double* partials;
  DevScalars* sc;
  int flex;
};

// The PCG update fused into the first pass: z += alpha p, r -= alpha q for the
// elements this block transforms, ||r||^2 accumulated, and the last block runs
// the convergence test of k_update_zr.  The pass then transforms the new r.
struct ZrFuse {
  double* z;
  double* r;
  const double* p;
  const double* q;
  double* partials;
  DevScalars* sc;
};

// tw[m] = (cos 2 pi m/N, sin 2 pi m/N), m < N/2;  dct[k] = (cos pi k/(2N), sin pi k/(2N)).
template <typename T, int N, int MODE, bool CONTIG, typename TI, typename TO, bool DOT = false,
          bool ZR = false>
__global__ void __launch_bounds__(256) k_fft(const TI* __restrict__ in, TO* __restrict__ out,
                                             const T* __restrict__ tw, const T* __restrict__ dct,
                                             long long inner, long long nlines, const DevScalars* sc,
                                             DotFuse df, ZrFuse zf) {
  if (sc != nullptr && sc->cg_done) return;
  using Sh = FftShape<T, N>;
  constexpr int CL = Sh::CL, LB = Sh::LB, NP = Sh::NP;
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf1 = buf0 + CL * NP;
  T* real1 = reinterpret_cast<T*>(buf1);  // [LB][NP] real staging in buf1
  cx<T>* tws = buf1 + CL * NP;            // twiddles, N/2
  cx<T>* dcs = tws + N / 2;               // DCT phases, N
  const int tid = threadIdx.x;
  for (int q = tid; q < N / 2; q += 256) tws[q] = cx<T>{tw[2 * q], tw[2 * q + 1]};
  if (MODE != FFT_DHT)
    for (int q = tid; q < N; q += 256) dcs[q] = cx<T>{dct[2 * q], dct[2 * q + 1]};
  const long long line0 = (long long)blockIdx.x * LB;
  const long long o = blockIdx.y;

  // ---- load LB real lines (with the fused z, r update when ZR).  A thread
  // takes its elements in batches whose loads are all issued before any of
  // them is used or stored, so one memory latency covers a batch.
  constexpr int PER = (LB * N + 255) / 256;        // elements per thread
  // (FP32 input: all of a thread's loads at once for N <= 512; the fused PCG
  // update moves four FP64 operands per element, so it takes 4 at a time)
  constexpr int BL = ZR ? (PER < 4 ? PER : 4) : (PER < 32 ? PER : 32);
  auto element = [&](int idx, int& l, int& i, long long& addr) -> bool {
    if (CONTIG) { l = idx / N; i = idx % N; } else { i = idx / LB; l = idx % LB; }
    const long long line = line0 + l;
    addr = CONTIG ? line * N + i : (o * N + i) * inner + line;
    return idx < LB * N && line < nlines;
  };
  auto stage = [&](int l, int i, T v) {
    if (MODE == FFT_DCT3) {
      real1[l * NP + i] = v;
    } else {
      const int p = (MODE == FFT_DCT2) ? ((i & 1) ? N - 1 - (i >> 1) : (i >> 1)) : i;
      T* dst = reinterpret_cast<T*>(&buf0[(l >> 1) * NP + swz<N>(p)]);
      dst[l & 1] = v;
    }
  };
  double rr = 0.0;
  const double alpha = ZR ? zf.sc->alpha : 0.0;
#pragma unroll 1
  for (int b0 = 0; b0 < PER; b0 += BL) {
    int ls[BL], is[BL];
    long long ad[BL];
    bool lv[BL];
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + 256 * (b0 + u);
      lv[u] = (b0 + u < PER) && element(idx, ls[u], is[u], ad[u]);
      if (!(idx < LB * N)) ls[u] = -1;
    }
    if constexpr (ZR) {
      double zv[BL], pv[BL], rv[BL], qv[BL];
#pragma unroll
      for (int u = 0; u < BL; ++u) {
        zv[u] = lv[u] ? zf.z[ad[u]] : 0.0;
        pv[u] = lv[u] ? zf.p[ad[u]] : 0.0;
        rv[u] = lv[u] ? zf.r[ad[u]] : 0.0;
        qv[u] = lv[u] ? zf.q[ad[u]] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < BL; ++u) {
        const double rn = fma(-alpha, qv[u], rv[u]);
        if (lv[u]) {
          zf.z[ad[u]] = fma(alpha, pv[u], zv[u]);
          zf.r[ad[u]] = rn;
        }
        rr = fma(rn, rn, rr);
        if (ls[u] >= 0) stage(ls[u], is[u], (T)rn);
      }
    } else {
      T v[BL];
#pragma unroll
      for (int u = 0; u < BL; ++u) v[u] = lv[u] ? (T)in[ad[u]] : T(0);
#pragma unroll
      for (int u = 0; u < BL; ++u)
        if (ls[u] >= 0) stage(ls[u], is[u], v[u]);
    }
  }
  __syncthreads();
  if (MODE == FFT_DCT3) {
    // W = exp(i th_k) (X_k - i X_{N-k}) with X = C/c, times 1/N of the inverse FFT.
    const T s0 = T(1) / sqrt(T(N)), s1 = T(1) / sqrt(T(2 * N));
    for (int idx = tid; idx < CL * N; idx += 256) {
      const int q = idx / N, k = idx % N;
      const T* xa = real1 + (2 * q) * NP;
      const T* xb = real1 + (2 * q + 1) * NP;
      const T sk = k == 0 ? s0 : s1, sm = s1;  // N-k > 0 whenever k > 0
      const T ak = xa[k] * sk, bk = xb[k] * sk;
      const T am = k == 0 ? T(0) : xa[N - k] * sm, bm = k == 0 ? T(0) : xb[N - k] * sm;
      const T c = dcs[k].x, s = dcs[k].y;
      const T war = c * ak + s * am, wai = s * ak - c * am;
      const T wbr = c * bk + s * bm, wbi = s * bk - c * bm;
      buf0[q * NP + swz<N>(k)] = cx<T>{war - wbi, wai + wbr};
    }
    __syncthreads();
  }

  // ---- Stockham FFT, one warp per complex line, natural order in and out:
  // for N >= 256 radix-8 stages (Ns = 1, 8, 64), then one radix-4 or radix-2
  // stage when log2 N is not a multiple of 3; for shorter lines radix-4 stages
  // and one radix-2 stage when log2 N is odd; in the mixed-radix Stockham formulation of
  // Govindaraju et al. (SC 2008): stage (R, Ns) reads v_r = src[j + r N/R],
  // twiddles v_r by exp(sgn 2 pi i r (j mod Ns) / (R Ns)), takes the R-point
  // DFT and writes dst[(j - j mod Ns) R + j mod Ns + r Ns].
  constexpr T sgn = (MODE == FFT_DCT3) ? T(1) : T(-1);
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int log2n = (N >= 512) ? 9 : (N >= 256) ? 8 : (N >= 128) ? 7 : (N >= 64) ? 6 : (N >= 32) ? 5 : (N >= 16) ? 4 : 3;
  constexpr bool R8 = FftRadix<N>::R8;
  // radix-8 schedule: n8 radix-8 stages, then radix 4 (r3 = 2) or 2 (r3 = 1);
  // radix-4 schedule: n4 radix-4 stages, then radix 2 when log2 N is odd
  constexpr int n8 = R8 ? log2n / 3 : 0, r3 = R8 ? log2n % 3 : 0;
  constexpr int n4 = R8 ? 0 : log2n / 2, n2 = R8 ? 0 : log2n % 2;
  // exp(sgn 2 pi i m / N) for 0 <= m < N from the half-circle table
  auto twid = [&](int m) -> cx<T> {
    const cx<T> t = tws[m & (N / 2 - 1)];
    const T f = (m & (N / 2)) ? T(-1) : T(1);
    return cx<T>{f * t.x, f * sgn * t.y};
  };
  auto cmul = [](cx<T> a, cx<T> w) { return cx<T>{a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x}; };
  auto add = [](cx<T> a, cx<T> b) { return cx<T>{a.x + b.x, a.y + b.y}; };
  auto sub = [](cx<T> a, cx<T> b) { return cx<T>{a.x - b.x, a.y - b.y}; };
  auto rot = [](cx<T> a) { return cx<T>{-sgn * a.y, sgn * a.x}; };  // times sgn i
  // 4-point DFT in place: B_s = sum_r b_r exp(sgn 2 pi i r s / 4)
  auto dft4 = [&](cx<T>& b0, cx<T>& b1, cx<T>& b2, cx<T>& b3) {
    const cx<T> s02 = add(b0, b2), d02 = sub(b0, b2), s13 = add(b1, b3), d13 = rot(sub(b1, b3));
    b0 = add(s02, s13);
    b1 = add(d02, d13);
    b2 = sub(s02, s13);
    b3 = sub(d02, d13);
  };
  const T h = T(0.70710678118654752440);  // cos(pi/4)
  for (int q = warp; q < CL; q += 8) {
    cx<T>* src = buf0 + q * NP;
    cx<T>* dst = buf1 + q * NP;
    int Ns = 1;
#pragma unroll
    for (int st = 0; st < n8; ++st, Ns <<= 3) {
#pragma unroll
      for (int j = lane; j < N / 8; j += 32) {
        const int k = j & (Ns - 1);
        const int m = k * (N / (8 * Ns));
        cx<T> a[8];
        a[0] = src[swz<N>(j)];
        if (st == 0) {  // Ns = 1: every twiddle is 1
#pragma unroll
          for (int r = 1; r < 8; ++r) a[r] = src[swz<N>(j + r * (N / 8))];
        } else {
#pragma unroll
          for (int r = 1; r < 8; ++r) a[r] = cmul(src[swz<N>(j + r * (N / 8))], twid(r * m));
        }
        // 8-point DFT: even and odd 4-point DFTs, then A_s = E_s + w^s O_s,
        // A_{s+4} = E_s - w^s O_s with w = exp(sgn 2 pi i / 8)
        dft4(a[0], a[2], a[4], a[6]);
        dft4(a[1], a[3], a[5], a[7]);
        const cx<T> o1{h * (a[3].x - sgn * a[3].y), h * (a[3].y + sgn * a[3].x)};
        const cx<T> o2 = rot(a[5]);
        const cx<T> o3{h * (-a[7].x - sgn * a[7].y), h * (-a[7].y + sgn * a[7].x)};
        const int d = ((j - k) << 3) + k;
        dst[swz<N>(d)] = add(a[0], a[1]);
        dst[swz<N>(d + 4 * Ns)] = sub(a[0], a[1]);
        dst[swz<N>(d + Ns)] = add(a[2], o1);
        dst[swz<N>(d + 5 * Ns)] = sub(a[2], o1);
        dst[swz<N>(d + 2 * Ns)] = add(a[4], o2);
        dst[swz<N>(d + 6 * Ns)] = sub(a[4], o2);
        dst[swz<N>(d + 3 * Ns)] = add(a[6], o3);
        dst[swz<N>(d + 7 * Ns)] = sub(a[6], o3);
      }
      __syncwarp();
      cx<T>* t = src; src = dst; dst = t;
    }
#pragma unroll
    for (int st = 0; st < n4; ++st, Ns <<= 2) {
#pragma unroll
      for (int j = lane; j < N / 4; j += 32) {
        const int k = j & (Ns - 1);
        const int m = k * (N / (4 * Ns));
        cx<T> a0 = src[swz<N>(j)];
        cx<T> a1 = src[swz<N>(j + N / 4)], a2 = src[swz<N>(j + N / 2)], a3 = src[swz<N>(j + 3 * N / 4)];
        if (st > 0) {  // Ns = 1 (the first stage): every twiddle is 1
          a1 = cmul(a1, twid(m));
          a2 = cmul(a2, twid(2 * m));
          a3 = cmul(a3, twid(3 * m));
        }
        dft4(a0, a1, a2, a3);
        const int d = ((j - k) << 2) + k;
        dst[swz<N>(d)] = a0;
        dst[swz<N>(d + Ns)] = a1;
        dst[swz<N>(d + 2 * Ns)] = a2;
        dst[swz<N>(d + 3 * Ns)] = a3;
      }
      __syncwarp();
      cx<T>* t = src; src = dst; dst = t;
    }
    if (r3 == 2) {
#pragma unroll
      for (int j = lane; j < N / 4; j += 32) {
        const int k = j & (Ns - 1);
        const int m = k * (N / (4 * Ns));
        cx<T> a0 = src[swz<N>(j)];
        cx<T> a1 = cmul(src[swz<N>(j + N / 4)], twid(m));
        cx<T> a2 = cmul(src[swz<N>(j + N / 2)], twid(2 * m));
        cx<T> a3 = cmul(src[swz<N>(j + 3 * N / 4)], twid(3 * m));
        dft4(a0, a1, a2, a3);
        const int d = ((j - k) << 2) + k;
        dst[swz<N>(d)] = a0;
        dst[swz<N>(d + Ns)] = a1;
        dst[swz<N>(d + 2 * Ns)] = a2;
        dst[swz<N>(d + 3 * Ns)] = a3;
      }
      __syncwarp();
    } else if (r3 == 1 || n2 == 1) {
#pragma unroll
      for (int j = lane; j < N / 2; j += 32) {
        const int k = j & (Ns - 1);
        const cx<T> a = src[swz<N>(j)];
        const cx<T> b = cmul(src[swz<N>(j + N / 2)], twid(k * (N / (2 * Ns))));
        const int d = ((j - k) << 1) + k;
        dst[swz<N>(d)] = add(a, b);
        dst[swz<N>(d + Ns)] = sub(a, b);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // stages taken: the result is in buf1 after an odd count
  const bool odd = ((n8 + n4 + ((r3 || n2) ? 1 : 0)) & 1) != 0;
  const cx<T>* Z = odd ? buf1 : buf0;
  T* R = reinterpret_cast<T*>(odd ? buf0 : buf1);  // real output staging [LB][NP]

  // ---- separate the packed pairs and finish the transform
  const T rsn = T(1) / sqrt(T(N));
  for (int idx = tid; idx < CL * N; idx += 256) {
    const int q = idx / N, k = idx % N;
    if (MODE == FFT_DCT3) {
      // x_{2n} = v_n, x_{2n+1} = v_{N-1-n}: walk the output position (k here)
      // so that the stores are contiguous; read v at the matching index
      const cx<T> zv = Z[q * NP + swz<N>((k & 1) ? N - 1 - (k >> 1) : (k >> 1))];
      R[(2 * q) * NP + k] = zv.x;
      R[(2 * q + 1) * NP + k] = zv.y;
    } else {
      const cx<T> zk = Z[q * NP + swz<N>(k)];
      const cx<T> zm = Z[q * NP + swz<N>((N - k) & (N - 1))];
      const T sr = T(0.5) * (zk.x + zm.x), si = T(0.5) * (zk.y - zm.y);  // X_a
      const T dr = T(0.5) * (zk.y + zm.y), di = T(0.5) * (zm.x - zk.x);  // X_b
      if (MODE == FFT_DHT) {
        R[(2 * q) * NP + k] = (sr - si) * rsn;
        R[(2 * q + 1) * NP + k] = (dr - di) * rsn;
      } else {
        const T ck = k == 0 ? T(1) / sqrt(T(N)) : sqrt(T(2) / T(N));
        const T c = dcs[k].x, s = dcs[k].y;
        R[(2 * q) * NP + k] = ck * (c * sr + s * si);
        R[(2 * q + 1) * NP + k] = ck * (c * dr + s * di);
      }
    }
  }
  __syncthreads();

  // ---- store (with the fused dot products of the PCG step when DOT; a
  // batch's dot operands are loaded before its stores)
  double a0 = 0.0, a1 = 0.0;
  constexpr int BS = DOT ? (PER < 8 ? PER : 8) : (PER < 16 ? PER : 16);
#pragma unroll 1
  for (int b0 = 0; b0 < PER; b0 += BS) {
    int ls[BS], is[BS];
    long long ad[BS];
    bool lv[BS];
#pragma unroll
    for (int u = 0; u < BS; ++u) {
      const int idx = tid + 256 * (b0 + u);
      lv[u] = (b0 + u < PER) && element(idx, ls[u], is[u], ad[u]);
    }
    double dr[DOT ? BS : 1], dq[DOT ? BS : 1];
    if constexpr (DOT) {
#pragma unroll
      for (int u = 0; u < BS; ++u) {
        dr[u] = lv[u] ? df.r[ad[u]] : 0.0;
        dq[u] = (lv[u] && df.flex) ? df.q[ad[u]] : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < BS; ++u) {
      if (lv[u]) {
        const TO v = (TO)R[ls[u] * NP + is[u]];
        out[ad[u]] = v;
        if constexpr (DOT) {
          a0 = fma(dr[u], (double)v, a0);
          a1 = fma(dq[u], (double)v, a1);
        }
      }
    }
  }
  if constexpr (ZR) {
    double part[1] = {rr};
    block_sum<1>(part);
    if (!publish_and_check_last<1>(part, zf.partials, &zf.sc->counter)) return;
    double tot[1];
    gather_partials<1>(zf.partials, tot);
    if (flat_tid() == 0) {
      DevScalars* s = zf.sc;
      s->rr = tot[0];
      s->cg_it += 1;
      const double tol = s->cg_tol;
      if (!isfinite(tot[0])) {
        s->cg_done = 1;
        if (s->status == MFG_OK) s->status = MFG_ERR_NONFINITE;
      } else if (tot[0] <= tol * tol * s->bnorm2) {
        s->cg_done = 1;
      } else if (s->cg_it >= s->max_cg) {
        s->cg_done = 1;
        if (s->status == MFG_OK) s->status = MFG_ERR_NOT_CONVERGED;
      }
      s->counter = 0;
    }
  }
  if constexpr (DOT) {
    double part[2] = {a0, a1};
    block_sum<2>(part);
    if (!publish_and_check_last<2>(part, df.partials, &df.sc->counter)) return;
    double tot[2];
    gather_partials<2>(df.partials, tot);
    if (flat_tid() == 0) {
      DevScalars* s = df.sc;
      const double rz_old = s->rz;
      s->qz = tot[1];
      s->beta = df.flex ? (-s->alpha * tot[1] / rz_old) : (tot[0] / rz_old);
      s->rz = tot[0];
      if (!isfinite(s->beta) || !(tot[0] > 0.0)) {
        s->cg_done = 1;
        if (s->status == MFG_OK) s->status = MFG_ERR_NONFINITE;
      }
      s->counter = 0;
    }
  }
}

bool fft_supported(int N) { return N >= 8 && N <= 512 && (N & (N - 1)) == 0; }

// Partial-sum slots the fused-dot y pass needs (2 per block).
long long fft_dot_partials(const Geom& g) {
  const long long lb = FftShape<float, 8>::LB;  // lines per block (same for every N and type)
  static_assert(FftShape<float, 8>::LB == FftShape<double, 512>::LB, "uniform lines per block");
  const long long nlines = g.n / g.ny;
  return 2 * ((nlines + lb - 1) / lb);
}

template <typename T, int N, int MODE, bool CONTIG, typename TI, typename TO, bool DOT = false,
          bool ZR = false>
static void launch_one(const TI* in, TO* out, const T* tw, const T* dct, long long inner,
                       long long outer, long long nlines, const DevScalars* sc, cudaStream_t s,
                       DotFuse df = DotFuse{}, ZrFuse zf = ZrFuse{}) {
  using Sh = FftShape<T, N>;
  dim3 grid((unsigned)((nlines + Sh::LB - 1) / Sh::LB), CONTIG ? 1u : (unsigned)outer);
  k_fft<T, N, MODE, CONTIG, TI, TO, DOT, ZR><<<grid, 256, Sh::smem, s>>>(in, out, tw, dct, inner, nlines, sc,
                                                                         df, zf);
}

template <typename T, int MODE, bool CONTIG, typename TI, typename TO, bool DOT = false,
          bool ZR = false>
static int set_attr_one() {
  int bad = 0;
#define MFG_FFT_ATTR(NN)                                                                      \
  bad |= cudaFuncSetAttribute(k_fft<T, NN, MODE, CONTIG, TI, TO, DOT, ZR>,                   \
                              cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                              (int)FftShape<T, NN>::smem) != cudaSuccess;
  MFG_FFT_ATTR(8) MFG_FFT_ATTR(16) MFG_FFT_ATTR(32) MFG_FFT_ATTR(64) MFG_FFT_ATTR(128)
  MFG_FFT_ATTR(256) MFG_FFT_ATTR(512)
#undef MFG_FFT_ATTR
  return bad;
}

template <typename T, int MODE, bool CONTIG, typename TI, typename TO, bool DOT = false,
          bool ZR = false>
static void dispatch(int N, const TI* in, TO* out, const T* tw, const T* dct, long long inner,
                     long long outer, long long nlines, const DevScalars* sc, cudaStream_t s,
                     DotFuse df = DotFuse{}, ZrFuse zf = ZrFuse{}) {
  switch (N) {
#define MFG_FFT_CASE(NN)                                                                              \
    case NN:                                                                                          \
      launch_one<T, NN, MODE, CONTIG, TI, TO, DOT, ZR>(in, out, tw, dct, inner, outer, nlines, sc, s, df, zf); \
      break;
    MFG_FFT_CASE(8) MFG_FFT_CASE(16) MFG_FFT_CASE(32) MFG_FFT_CASE(64) MFG_FFT_CASE(128) MFG_FFT_CASE(256)
#undef MFG_FFT_CASE
    default:
      launch_one<T, 512, MODE, CONTIG, TI, TO, DOT, ZR>(in, out, tw, dct, inner, outer, nlines, sc, s, df, zf);
      break;
  }
}

// y axis (contiguous), first pass: FP64 residual in, T out; with zr != nullptr
// the PCG update z += alpha p, r -= alpha q and its convergence test come first.
template <typename T>
void fft_y_forward(int N, int periodic, const double* in, T* out, const T* tw, const T* dct,
                   long long nlines, const DevScalars* sc, cudaStream_t s, const PcgZr* zr) {
  if (zr) {
    ZrFuse zf{zr->z, zr->r, zr->p, zr->q, zr->partials, zr->sc};
    if (periodic)
      dispatch<T, FFT_DHT, true, double, T, false, true>(N, in, out, tw, dct, 1, 1, nlines, sc, s, DotFuse{}, zf);
    else
      dispatch<T, FFT_DCT2, true, double, T, false, true>(N, in, out, tw, dct, 1, 1, nlines, sc, s, DotFuse{}, zf);
    return;
  }
  if (periodic)
    dispatch<T, FFT_DHT, true, double, T>(N, in, out, tw, dct, 1, 1, nlines, sc, s);
  else
    dispatch<T, FFT_DCT2, true, double, T>(N, in, out, tw, dct, 1, 1, nlines, sc, s);
}
// y axis, last pass: T in, FP64 out; with dot != nullptr the PCG dot products
// (r.zp, q.zp, beta) are fused into the store.
template <typename T>
void fft_y_inverse(int N, int periodic, const T* in, double* out, const T* tw, const T* dct,
                   long long nlines, const DevScalars* sc, cudaStream_t s, const PcgDot* dot) {
  if (dot) {
    DotFuse df{dot->r, dot->q, dot->partials, dot->sc, dot->flex};
    if (periodic)
      dispatch<T, FFT_DHT, true, T, double, true>(N, in, out, tw, dct, 1, 1, nlines, sc, s, df);
    else
      dispatch<T, FFT_DCT3, true, T, double, true>(N, in, out, tw, dct, 1, 1, nlines, sc, s, df);
    return;
  }
  if (periodic)
    dispatch<T, FFT_DHT, true, T, double>(N, in, out, tw, dct, 1, 1, nlines, sc, s);
  else
    dispatch<T, FFT_DCT3, true, T, double>(N, in, out, tw, dct, 1, 1, nlines, sc, s);
}
// x axis (stride ny), both directions.
template <typename T>
void fft_x(int N, int periodic, int inverse, const T* in, T* out, const T* tw, const T* dct,
           long long inner, long long outer, const DevScalars* sc, cudaStream_t s) {
  if (periodic)
    dispatch<T, FFT_DHT, false, T, T>(N, in, out, tw, dct, inner, outer, inner, sc, s);
  else if (!inverse)
    dispatch<T, FFT_DCT2, false, T, T>(N, in, out, tw, dct, inner, outer, inner, sc, s);
  else
    dispatch<T, FFT_DCT3, false, T, T>(N, in, out, tw, dct, inner, outer, inner, sc, s);
}

template void fft_y_forward<float>(int, int, const double*, float*, const float*, const float*, long long,
                                   const DevScalars*, cudaStream_t, const PcgZr*);
template void fft_y_forward<double>(int, int, const double*, double*, const double*, const double*, long long,
                                    const DevScalars*, cudaStream_t, const PcgZr*);
template void fft_y_inverse<float>(int, int, const float*, double*, const float*, const float*, long long,
                                   const DevScalars*, cudaStream_t, const PcgDot*);
template void fft_y_inverse<double>(int, int, const double*, double*, const double*, const double*, long long,
                                    const DevScalars*, cudaStream_t, const PcgDot*);
template void fft_x<float>(int, int, int, const float*, float*, const float*, const float*, long long, long long,
                           const DevScalars*, cudaStream_t);
template void fft_x<double>(int, int, int, const double*, double*, const double*, const double*, long long,
                            long long, const DevScalars*, cudaStream_t);

int fft_configure() {
  int bad = 0;
  bad |= set_attr_one<float, FFT_DHT, true, double, float>();
  bad |= set_attr_one<float, FFT_DCT2, true, double, float>();
  bad |= set_attr_one<float, FFT_DHT, true, float, double>();
  bad |= set_attr_one<float, FFT_DCT3, true, float, double>();
  bad |= set_attr_one<float, FFT_DHT, true, float, double, true>();
  bad |= set_attr_one<float, FFT_DCT3, true, float, double, true>();
  bad |= set_attr_one<double, FFT_DHT, true, double, double, true>();
  bad |= set_attr_one<double, FFT_DCT3, true, double, double, true>();
  bad |= set_attr_one<float, FFT_DHT, true, double, float, false, true>();
  bad |= set_attr_one<float, FFT_DCT2, true, double, float, false, true>();
  bad |= set_attr_one<double, FFT_DHT, true, double, double, false, true>();
  bad |= set_attr_one<double, FFT_DCT2, true, double, double, false, true>();
  bad |= set_attr_one<float, FFT_DHT, false, float, float>();
  bad |= set_attr_one<float, FFT_DCT2, false, float, float>();
  bad |= set_attr_one<float, FFT_DCT3, false, float, float>();
  bad |= set_attr_one<double, FFT_DHT, true, double, double>();
  bad |= set_attr_one<double, FFT_DCT2, true, double, double>();
  bad |= set_attr_one<double, FFT_DCT3, true, double, double>();
  bad |= set_attr_one<double, FFT_DHT, false, double, double>();
  bad |= set_attr_one<double, FFT_DCT2, false, double, double>();
  bad |= set_attr_one<double, FFT_DCT3, false, double, double>();
  return bad ? MFG_ERR_CUDA : MFG_OK;
}

}  // namespace mfg
