// Spatial passes of the preconditioner by FFT, for axis lengths that are powers
// of two (Alg. 2 lines 12-16: transform along y, then x, divide, invert).
//
// One block takes LB real lines of length N (rows of the contiguous y axis, or
// columns of the x axis), packs them pairwise into CL = LB/2 complex lines
// z = x_a + i x_b, runs a radix-2 Stockham FFT per complex line in shared
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

namespace mfg {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T x, y;
};

enum { FFT_DHT = 0, FFT_DCT2 = 1, FFT_DCT3 = 2 };

template <typename T, int N>
struct FftShape {
  static constexpr int CL = (sizeof(T) == 8 && N > 256) ? 8 : 16;  // complex lines per block
  static constexpr int LB = 2 * CL;                                 // real lines per block
  static constexpr size_t smem = 2 * (size_t)CL * N * sizeof(cx<T>);
};

// tw[m] = (cos 2 pi m/N, sin 2 pi m/N), m < N/2;  dct[k] = (cos pi k/(2N), sin pi k/(2N)).
template <typename T, int N, int MODE, bool CONTIG, typename TI, typename TO>
__global__ void __launch_bounds__(256) k_fft(const TI* __restrict__ in, TO* __restrict__ out,
                                             const T* __restrict__ tw, const T* __restrict__ dct,
                                             long long inner, long long nlines, const DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  using Sh = FftShape<T, N>;
  constexpr int CL = Sh::CL, LB = Sh::LB;
  extern __shared__ unsigned char smem_raw[];
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf1 = buf0 + CL * N;
  T* real1 = reinterpret_cast<T*>(buf1);  // [LB][N] real staging in buf1
  const int tid = threadIdx.x;
  const long long line0 = (long long)blockIdx.x * LB;
  const long long o = blockIdx.y;

  // ---- load LB real lines
  for (int idx = tid; idx < LB * N; idx += 256) {
    int l, i;
    if (CONTIG) { l = idx / N; i = idx % N; } else { i = idx / LB; l = idx % LB; }
    const long long line = line0 + l;
    T v = T(0);
    if (line < nlines) {
      const long long addr = CONTIG ? line * N + i : (o * N + i) * inner + line;
      v = (T)in[addr];
    }
    if (MODE == FFT_DCT3) {
      real1[l * N + i] = v;
    } else {
      const int p = (MODE == FFT_DCT2) ? ((i & 1) ? N - 1 - (i >> 1) : (i >> 1)) : i;
      T* dst = reinterpret_cast<T*>(&buf0[(l >> 1) * N + p]);
      dst[l & 1] = v;
    }
  }
  __syncthreads();
  if (MODE == FFT_DCT3) {
    // W = exp(i th_k) (X_k - i X_{N-k}) with X = C/c, times 1/N of the inverse FFT.
    const T s0 = T(1) / sqrt(T(N)), s1 = T(1) / sqrt(T(2 * N));
    for (int idx = tid; idx < CL * N; idx += 256) {
      const int q = idx / N, k = idx % N;
      const T* xa = real1 + (2 * q) * N;
      const T* xb = real1 + (2 * q + 1) * N;
      const T sk = k == 0 ? s0 : s1, sm = s1;  // N-k > 0 whenever k > 0
      const T ak = xa[k] * sk, bk = xb[k] * sk;
      const T am = k == 0 ? T(0) : xa[N - k] * sm, bm = k == 0 ? T(0) : xb[N - k] * sm;
      const T c = dct[2 * k], s = dct[2 * k + 1];
      const T war = c * ak + s * am, wai = s * ak - c * am;
      const T wbr = c * bk + s * bm, wbi = s * bk - c * bm;
      buf0[q * N + k] = cx<T>{war - wbi, wai + wbr};
    }
    __syncthreads();
  }

  // ---- radix-2 Stockham FFT, one warp per complex line
  constexpr T sgn = (MODE == FFT_DCT3) ? T(1) : T(-1);
  const int warp = tid >> 5, lane = tid & 31;
  int log2n = 0;
  for (int t = N; t > 1; t >>= 1) ++log2n;
  for (int q = warp; q < CL; q += 8) {
    cx<T>* src = buf0 + q * N;
    cx<T>* dst = buf1 + q * N;
    for (int Ns = 1; Ns < N; Ns <<= 1) {
      for (int j = lane; j < N / 2; j += 32) {
        const int k = j & (Ns - 1);
        const int m = k * (N / (2 * Ns));
        const T wc = tw[2 * m], ws = sgn * tw[2 * m + 1];
        const cx<T> a = src[j];
        const cx<T> b0 = src[j + N / 2];
        const cx<T> b{b0.x * wc - b0.y * ws, b0.x * ws + b0.y * wc};
        const int d = ((j - k) << 1) + k;
        dst[d] = cx<T>{a.x + b.x, a.y + b.y};
        dst[d + Ns] = cx<T>{a.x - b.x, a.y - b.y};
      }
      __syncwarp();
      cx<T>* t = src; src = dst; dst = t;
    }
  }
  __syncthreads();
  const cx<T>* Z = (log2n & 1) ? buf1 : buf0;
  T* R = reinterpret_cast<T*>((log2n & 1) ? buf0 : buf1);  // real output staging [LB][N]

  // ---- separate the packed pairs and finish the transform
  const T rsn = T(1) / sqrt(T(N));
  for (int idx = tid; idx < CL * N; idx += 256) {
    const int q = idx / N, k = idx % N;
    const cx<T> zk = Z[q * N + k];
    if (MODE == FFT_DCT3) {
      const int pos = (k < N / 2) ? 2 * k : 2 * (N - 1 - k) + 1;
      R[(2 * q) * N + pos] = zk.x;
      R[(2 * q + 1) * N + pos] = zk.y;
    } else {
      const cx<T> zm = Z[q * N + ((N - k) & (N - 1))];
      const T sr = T(0.5) * (zk.x + zm.x), si = T(0.5) * (zk.y - zm.y);  // X_a
      const T dr = T(0.5) * (zk.y + zm.y), di = T(0.5) * (zm.x - zk.x);  // X_b
      if (MODE == FFT_DHT) {
        R[(2 * q) * N + k] = (sr - si) * rsn;
        R[(2 * q + 1) * N + k] = (dr - di) * rsn;
      } else {
        const T ck = k == 0 ? T(1) / sqrt(T(N)) : sqrt(T(2) / T(N));
        const T c = dct[2 * k], s = dct[2 * k + 1];
        R[(2 * q) * N + k] = ck * (c * sr + s * si);
        R[(2 * q + 1) * N + k] = ck * (c * dr + s * di);
      }
    }
  }
  __syncthreads();

  // ---- store
  for (int idx = tid; idx < LB * N; idx += 256) {
    int l, i;
    if (CONTIG) { l = idx / N; i = idx % N; } else { i = idx / LB; l = idx % LB; }
    const long long line = line0 + l;
    if (line < nlines) {
      const long long addr = CONTIG ? line * N + i : (o * N + i) * inner + line;
      out[addr] = (TO)R[l * N + i];
    }
  }
}

bool fft_supported(int N) { return N >= 8 && N <= 512 && (N & (N - 1)) == 0; }

template <typename T, int N, int MODE, bool CONTIG, typename TI, typename TO>
static void launch_one(const TI* in, TO* out, const T* tw, const T* dct, long long inner,
                       long long outer, long long nlines, const DevScalars* sc, cudaStream_t s) {
  using Sh = FftShape<T, N>;
  dim3 grid((unsigned)((nlines + Sh::LB - 1) / Sh::LB), CONTIG ? 1u : (unsigned)outer);
  k_fft<T, N, MODE, CONTIG, TI, TO><<<grid, 256, Sh::smem, s>>>(in, out, tw, dct, inner, nlines, sc);
}

template <typename T, int MODE, bool CONTIG, typename TI, typename TO>
static int set_attr_one() {
  int bad = 0;
#define MFG_FFT_ATTR(NN)                                                                      \
  bad |= cudaFuncSetAttribute(k_fft<T, NN, MODE, CONTIG, TI, TO>,                            \
                              cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                              (int)FftShape<T, NN>::smem) != cudaSuccess;
  MFG_FFT_ATTR(8) MFG_FFT_ATTR(16) MFG_FFT_ATTR(32) MFG_FFT_ATTR(64) MFG_FFT_ATTR(128)
  MFG_FFT_ATTR(256) MFG_FFT_ATTR(512)
#undef MFG_FFT_ATTR
  return bad;
}

template <typename T, int MODE, bool CONTIG, typename TI, typename TO>
static void dispatch(int N, const TI* in, TO* out, const T* tw, const T* dct, long long inner,
                     long long outer, long long nlines, const DevScalars* sc, cudaStream_t s) {
  switch (N) {
    case 8: launch_one<T, 8, MODE, CONTIG, TI, TO>(in, out, tw, dct, inner, outer, nlines, sc, s); break;
    case 16: launch_one<T, 16, MODE, CONTIG, TI, TO>(in, out, tw, dct, inner, outer, nlines, sc, s); break;
    case 32: launch_one<T, 32, MODE, CONTIG, TI, TO>(in, out, tw, dct, inner, outer, nlines, sc, s); break;
    case 64: launch_one<T, 64, MODE, CONTIG, TI, TO>(in, out, tw, dct, inner, outer, nlines, sc, s); break;
    case 128: launch_one<T, 128, MODE, CONTIG, TI, TO>(in, out, tw, dct, inner, outer, nlines, sc, s); break;
    case 256: launch_one<T, 256, MODE, CONTIG, TI, TO>(in, out, tw, dct, inner, outer, nlines, sc, s); break;
    default: launch_one<T, 512, MODE, CONTIG, TI, TO>(in, out, tw, dct, inner, outer, nlines, sc, s); break;
  }
}

// y axis (contiguous), first pass: FP64 residual in, T out.
template <typename T>
void fft_y_forward(int N, int periodic, const double* in, T* out, const T* tw, const T* dct,
                   long long nlines, const DevScalars* sc, cudaStream_t s) {
  if (periodic)
    dispatch<T, FFT_DHT, true, double, T>(N, in, out, tw, dct, 1, 1, nlines, sc, s);
  else
    dispatch<T, FFT_DCT2, true, double, T>(N, in, out, tw, dct, 1, 1, nlines, sc, s);
}
// y axis, last pass: T in, FP64 out.
template <typename T>
void fft_y_inverse(int N, int periodic, const T* in, double* out, const T* tw, const T* dct,
                   long long nlines, const DevScalars* sc, cudaStream_t s) {
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
                                   const DevScalars*, cudaStream_t);
template void fft_y_forward<double>(int, int, const double*, double*, const double*, const double*, long long,
                                    const DevScalars*, cudaStream_t);
template void fft_y_inverse<float>(int, int, const float*, double*, const float*, const float*, long long,
                                   const DevScalars*, cudaStream_t);
template void fft_y_inverse<double>(int, int, const double*, double*, const double*, const double*, long long,
                                    const DevScalars*, cudaStream_t);
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
