// mfg_apply_precond_noalloc: the preconditioner apply z = P^{-1} r without a
// plan and without any device allocation.
//
// Who needs it: code that must not allocate device memory at the point of
// the call, for example work recorded into a CUDA graph under global capture
// (cudaMalloc is not allowed there), callers whose memory is owned by a pool
// or a framework allocator they cannot bypass, or real-time paths where an
// allocation's latency or possible failure is unacceptable.  Such callers
// cannot build an mfg_plan (it allocates tables and workspace), so this entry
// point derives everything from the problem description.
//
// Where its memory comes from: one file-scope __device__ array, sized for the
// limits below and resident on every GPU that loads the library until the
// process exits.  The transform tables and the two ping-pong work buffers of
// the preconditioner passes are carved out of it.  All calls share it, so two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race; calls on one stream are ordered and safe.  Nothing is
// assumed to be zero: every call rewrites the tables and both work buffers
// are fully written before they are read.
#include <atomic>
#include <cmath>
#include <string>

#include "mfg_internal.cuh"

namespace mfg {
namespace {

constexpr long long kNaMaxN = 1LL << 18;  // space-time points n = N_t * Nx * Ny
constexpr int kNaMaxAxis = 256;           // points per spatial axis
constexpr int kNaMaxNt = 128;             // time steps
constexpr size_t kNaWork = 2 * (size_t)kNaMaxN;
constexpr size_t kNaH = (size_t)kNaMaxAxis * kNaMaxAxis;
constexpr size_t kNaV = (size_t)kNaMaxNt * kNaMaxNt;
constexpr size_t kNaS = (size_t)kNaMaxAxis * kNaMaxAxis;
// FFT twiddles of a power-of-two axis: N/2 complex (cos, sin)(2 pi m/N) and N
// complex (cos, sin)(pi k/(2N)), i.e. 3N values per axis
constexpr size_t kNaTw = 3 * (size_t)kNaMaxAxis;
constexpr size_t kNaDoubles = kNaWork + 2 * kNaH + kNaV + kNaMaxNt + 2 * kNaS + 2 * kNaTw;  // 6.4 MB

__device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

// Device address of g_noalloc_scratch per device, resolved by the first call
// on that device.  Atomic, so first calls from several host threads at once
// are well defined (each resolves the same address).
constexpr int kMaxDevices = 64;
std::atomic<void*> g_noalloc_ptr[kMaxDevices];

__device__ double axis_lambda(int a, int N, int per) {
  if (N == 1) return 0.0;
  return 2.0 - 2.0 * cospi((per ? 2.0 : 1.0) * a / N);
}

// Twiddles of the FFT spatial passes for a power-of-two axis of length N
// (same definitions as the plan's): tw[m] = (cos, sin)(2 pi m/N), m < N/2;
// dct[k] = (cos, sin)(pi k/(2N)), k < N; interleaved (cos, sin) pairs.
template <typename T>
__device__ void fft_twiddle(long long q, int N, T* tw, T* dct) {
  if (q < N) {
    const int m = (int)(q >> 1);
    tw[q] = (T)((q & 1) ? sinpi(2.0 * m / N) : cospi(2.0 * m / N));
  } else {
    q -= N;
    const int k = (int)(q >> 1);
    dct[q] = (T)((q & 1) ? sinpi(k / (2.0 * N)) : cospi(k / (2.0 * N)));
  }
}

// Fills the tables of eq. pstrec (same definitions as the plan's host tables:
// Hartley / DCT-II in space, DCT-VIII / DST-I in time, Lambda_1, Lambda_2, and
// the FFT twiddles of power-of-two axes; twx/twy null otherwise), evaluated on
// the device with cospi/sinpi.
template <typename T>
__global__ void k_noalloc_tables(Geom g, int l, T* Hx, T* Hy, T* V, T* lamt, T* L1, T* L2, T* twx, T* dctx,
                                 T* twy, T* dcty) {
  const long long nHx = (long long)g.nx * g.nx, nHy = (long long)g.ny * g.ny;
  const long long nV = (long long)g.nt * g.nt;
  const long long nTx = twx ? 3LL * g.nx : 0, nTy = twy ? 3LL * g.ny : 0;
  const long long total = nHx + nHy + nV + g.nt + g.S + nTx + nTy;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long q = e;
    if (q >= total - nTx - nTy) {
      q -= total - nTx - nTy;
      if (q < nTx)
        fft_twiddle(q, g.nx, twx, dctx);
      else
        fft_twiddle(q - nTx, g.ny, twy, dcty);
      continue;
    }
    if (q < nHx + nHy) {
      const bool xa = q < nHx;
      const int N = xa ? g.nx : g.ny, per = xa ? g.perx : g.pery;
      if (!xa) q -= nHx;
      const int a = (int)(q / N), b = (int)(q % N);
      double h;
      if (N == 1) {
        h = 1.0;
      } else if (per) {
        const double th = 2.0 * (double)(((long long)a * b) % N) / N;  // angle / pi
        h = (cospi(th) + sinpi(th)) / sqrt((double)N);
      } else {
        const double ca = a == 0 ? sqrt(1.0 / N) : sqrt(2.0 / N);
        h = ca * cospi(a * (2.0 * b + 1.0) / (2.0 * N));
      }
      (xa ? Hx : Hy)[q] = (T)h;
      continue;
    }
    q -= nHx + nHy;
    const int N = g.nt;
    if (q < nV) {
      const int k = (int)(q / N), j = (int)(q % N);
      const double v = (l == 1)
                           ? 2.0 / sqrt(2.0 * N + 1.0) * cospi((2.0 * k + 1.0) * (2.0 * j + 1.0) / (2.0 * (2.0 * N + 1.0)))
                           : sqrt(2.0 / (N + 1.0)) * sinpi((j + 1.0) * (k + 1.0) / (N + 1.0));
      V[q] = (T)v;
      continue;
    }
    q -= nV;
    if (q < N) {
      const int k = (int)q;
      lamt[k] = (T)((l == 1) ? 2.0 - 2.0 * cospi((k + 0.5) / (N + 0.5)) : 2.0 - 2.0 * cospi((k + 1.0) / (N + 1.0)));
      continue;
    }
    q -= N;
    const int a = (int)(q / g.ny), b = (int)(q % g.ny);
    const double D = axis_lambda(a, g.nx, g.perx) * g.ax + axis_lambda(b, g.ny, g.pery) * g.ay;
    L1[q] = (T)(g.nu * g.nu * D * D + 2.0 * D);
    L2[q] = (T)((g.nu * D + g.idt) * g.idt);
  }
}

template <typename T>
void carve(double* base, const Geom& g, PrecTables* t, T** w0) {
  T* p = reinterpret_cast<T*>(base);
  *w0 = p;
  p += kNaWork;
  T* Hx = p; p += kNaH;
  T* Hy = p; p += kNaH;
  T* V = p; p += kNaV;
  T* lamt = p; p += kNaMaxNt;
  T* L1 = p; p += kNaS;
  T* L2 = p; p += kNaS;
  T* twx = p; T* dctx = p + kNaMaxAxis; p += kNaTw;
  T* twy = p; T* dcty = p + kNaMaxAxis;
  const bool fx = g.nx > 1 && fft_supported(g.nx), fy = fft_supported(g.ny);
  if (!fx) twx = dctx = nullptr;
  if (!fy) twy = dcty = nullptr;
  if constexpr (sizeof(T) == 8) {
    t->Hx64 = Hx; t->Hy64 = Hy; t->Vt64 = V; t->lamt64 = lamt; t->L1_64 = L1; t->L2_64 = L2;
    t->twx64 = twx; t->dctx64 = dctx; t->twy64 = twy; t->dcty64 = dcty;
  } else {
    t->Hx32 = Hx; t->Hy32 = Hy; t->Vt32 = V; t->lamt32 = lamt; t->L1_32 = L1; t->L2_32 = L2;
    t->twx32 = twx; t->dctx32 = dctx; t->twy32 = twy; t->dcty32 = dcty;
  }
  t->nx = g.nx; t->ny = g.ny; t->nt = g.nt;
}

}  // namespace
}  // namespace mfg

using namespace mfg;

extern "C" int mfg_apply_precond_noalloc(const mfg_problem* p, const double* r, double* z,
                                         void* stream) {
  if (!p || !r || !z || r == z)
    return set_error(MFG_ERR_INVALID_ARG, "problem, r and z must be non-null and r != z");
  int rc = validate_problem(*p, 0);
  if (rc != MFG_OK) return rc;
  if (p->l == 0)
    return set_error(MFG_ERR_UNSUPPORTED, "mfg_apply_precond_noalloc: l = 0 needs plan-built factors");
  if (p->nu_field != nullptr)
    return set_error(MFG_ERR_UNSUPPORTED, "mfg_apply_precond_noalloc: a viscosity field needs plan-built factors");
  const Geom g = make_geom(*p);
  if (g.n > kNaMaxN || g.nx > kNaMaxAxis || g.ny > kNaMaxAxis || g.nt > kNaMaxNt)
    return set_error(MFG_ERR_INVALID_ARG,
                     "mfg_apply_precond_noalloc: problem exceeds its static scratch (limits: "
                     "N_t*Nx*Ny <= 262144, Nx, Ny <= 256, N_t <= 128)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error(MFG_ERR_CUDA, "mfg_apply_precond_noalloc: no usable current device");
  void* cached = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (cached == nullptr) {
    // First call on this device: resolve the device address of the static
    // scratch (its host-side name is not a device address) and set the kernel
    // attributes the preconditioner passes need.
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr)
      return set_error(MFG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    if (precond_configure() != MFG_OK)
      return set_error(MFG_ERR_CUDA, "cudaFuncSetAttribute failed");
    g_noalloc_ptr[dev].store(ptr, std::memory_order_release);
    cached = ptr;
  }
  double* base = static_cast<double*>(cached);
  cudaStream_t s = (cudaStream_t)stream;
  PrecTables t{};
  const long long ntab = (long long)g.nx * g.nx + (long long)g.ny * g.ny + (long long)g.nt * g.nt + g.nt + g.S +
                         3LL * (g.nx + g.ny);
  const int nb = (int)std::min<long long>((ntab + kThreads - 1) / kThreads, 1024);
  if (p->precision != MFG_FP64) {
    // FP32 transforms; MFG_MIXED_TC takes the tensor-core time pass as in the
    // plan, MFG_MIXED_DF (which differs from MFG_MIXED only in the AAt stencil)
    // runs as MFG_MIXED
    float* w0 = nullptr;
    carve<float>(base, g, &t, &w0);
    k_noalloc_tables<float><<<nb, kThreads, 0, s>>>(g, p->l, t.Hx32, t.Hy32, t.Vt32, t.lamt32, t.L1_32, t.L2_32,
                                                     t.twx32, t.dctx32, t.twy32, t.dcty32);
    launch_precond(g, t, p->precision == MFG_MIXED_TC ? MFG_MIXED_TC : MFG_MIXED, r, z, nullptr, w0, nullptr, s);
  } else {
    double* w0 = nullptr;
    carve<double>(base, g, &t, &w0);
    k_noalloc_tables<double><<<nb, kThreads, 0, s>>>(g, p->l, t.Hx64, t.Hy64, t.Vt64, t.lamt64, t.L1_64,
                                                      t.L2_64, t.twx64, t.dctx64, t.twy64, t.dcty64);
    launch_precond(g, t, MFG_FP64, r, z, w0, nullptr, nullptr, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(MFG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return MFG_OK;
}
