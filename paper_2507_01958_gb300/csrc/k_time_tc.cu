// Time pass of the preconditioner on the 5th-generation tensor cores
// (tcgen05, TF32), the MFG_MIXED_TC precision: per spatial mode s,
//   Y[:, s] = V X[:, s],   Y[r, s] /= Lambda_1(s) + lambda_r Lambda_2(s),
//   out[:, s] = V^T Y[:, s]                                   (eq. pstrec)
// with V the orthonormal DCT-VIII (l = 1) or DST-I (l = 2) matrix of Sec. 4.2
// (symmetric, checked on the host, so V^T = V).
//
// Both products are dense N_t x N_t contractions over a strip of TW = 128
// spatial modes, issued as D = A B with
//   A = X^T (M = TW modes x K = N_t times),  B = V (N = N_t x K = N_t),
// so the accumulator D[s][r] sits in tensor memory with one spatial mode per
// TMEM lane: the division by S(r, s) is per thread and the final stores are
// coalesced along s.  One elected thread issues the MMAs; completion is
// signalled through an mbarrier (tcgen05.commit) whose waits are bounded.
//
// Precision: each FP32 operand x is split as x = hi + lo with hi = x rounded
// towards zero to TF32 (10 mantissa bits) and lo = x - hi (exact in FP32);
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi ("3xTF32").  The dropped A_lo B_lo
// term and the TF32 rounding of lo leave a relative error of ~2^-20 per
// product, near the FP32 path's.
//
// Operands live in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices (128 contiguous bytes), core matrices
// adjacent in K one leading-byte-offset (LBO) apart, 8-row groups 128 bytes
// apart (the stride-byte-offset, SBO).  For an operand with R rows:
//   byte(row, k) = (k / 4) * 16 R + (row / 8) * 128 + (row % 8) * 16 + (k % 4) * 4,
// LBO = 16 R, SBO = 128; one MMA (K = 8) spans two core matrices in K.
#include <cstdint>

#include "mfg_internal.cuh"

namespace mfg {
namespace {

constexpr int kTcTW = 128;      // spatial modes per strip (the MMA's M)
constexpr int kTcThreads = 256;
constexpr uint32_t kTcPolls = 1u << 20;  // mbarrier polls before a wait gives up
// Poll limit under the fault-injection hook (no MMA issued, nothing ever
// arrives): short, so the test of the timeout path costs milliseconds.
constexpr uint32_t kTcPollsInjected = 1u << 12;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, LBO and SBO in
// 16-byte units, descriptor version 1 (bits 46-47), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// tcgen05 instruction descriptor for kind::tf32: D in F32 (bits 4-5 = 1),
// A and B in TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the given phase parity of an mbarrier, giving up after `polls` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t polls) {
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

// 16 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

__device__ __forceinline__ void split4(const float (&x)[4], float4& hi, float4& lo) {
  tf32_split(x[0], hi.x, lo.x);
  tf32_split(x[1], hi.y, lo.y);
  tf32_split(x[2], hi.z, lo.z);
  tf32_split(x[3], hi.w, lo.w);
}

template <int NT>
struct TcShape {
  static constexpr int TW = kTcTW;
  static constexpr int KC = NT < 64 ? NT : 64;  // K (time) columns of A staged per round
  static constexpr int NKC = NT / KC;           // staging rounds per product
  static constexpr uint32_t LBO_A = 16u * TW, LBO_B = 16u * NT, SBO = 128u;
  static constexpr uint32_t NCOLS = 2u * NT;    // two F32 accumulators of N_t columns
  static constexpr size_t floats = 2u * TW * KC + 2u * NT * NT + 2u * TW + NT;
  static constexpr size_t smem = floats * 4;
  // Shared memory limits the blocks per SM to 1 (N_t = 128), 2 (64) or 5 (32),
  // so the tensor-memory columns of the resident blocks (NCOLS each) never
  // exceed the SM's 512, even with blocks of other N_t beside them.
  static_assert((228u * 1024u / (smem + 1024u)) * NCOLS <= 512u, "TMEM columns of co-resident blocks");
};

template <int NT>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_time_tc(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ V,
              const float* __restrict__ lamt, const float* __restrict__ L1, const float* __restrict__ L2,
              int S, DevScalars* sc) {
  if (sc != nullptr && sc->cg_done) return;
  // Fault-injection hook (MFG_INJECT_TC_NO_COMMIT): the elected thread issues
  // neither the MMAs nor their commit, so no tensor-core work is ever in flight
  // and the bounded completion wait must run out.
  const bool no_commit = sc != nullptr && sc->inject == MFG_INJECT_TC_NO_COMMIT;
  const uint32_t polls = no_commit ? kTcPollsInjected : kTcPolls;
  using Sh = TcShape<NT>;
  constexpr int TW = Sh::TW, KC = Sh::KC, NKC = Sh::NKC, HALF = NT / 2;
  constexpr uint32_t LBO_A = Sh::LBO_A, LBO_B = Sh::LBO_B, SBO = Sh::SBO, NCOLS = Sh::NCOLS;
  constexpr uint32_t IDESC = tc_idesc_tf32(TW, NT);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* Ahi = reinterpret_cast<float*>(smem_raw);
  float* Alo = Ahi + TW * KC;
  float* Bhi = Alo + TW * KC;
  float* Blo = Bhi + NT * NT;
  float* L1s = Blo + NT * NT;
  float* L2s = L1s + TW;
  float* lams = L2s + TW;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mb = smem_u32(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // V -> B operand (hi, lo): row n = output time, k = input time, V row-major.
  for (int q = tid; q < NT * NT / 4; q += kTcThreads) {
    const int n = q / (NT / 4), kq = q % (NT / 4);
    const float4 v4 = reinterpret_cast<const float4*>(V)[q];
    const float x[4] = {v4.x, v4.y, v4.z, v4.w};
    float4 h, l;
    split4(x, h, l);
    const uint32_t off = kq * LBO_B + (n >> 3) * 128u + (n & 7) * 16u;
    *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Bhi) + off) = h;
    *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Blo) + off) = l;
  }
  for (int q = tid; q < NT; q += kTcThreads) lams[q] = lamt[q];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t d1 = tmem, d2 = tmem + (uint32_t)NT;  // accumulator column bases
  const int sub = warp & 3;                             // TMEM lane quarter of this warp
  const int half = warp >> 2;                           // accumulator columns [half*NT/2, +NT/2)
  const int m = sub * 32 + lane;                        // strip row (spatial mode) of this thread
  const uint32_t lane_bits = (uint32_t)(sub * 32) << 16;
  const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo), b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
  uint32_t parity = 0;
  bool failed = false;
  const int nstrips = (S + TW - 1) / TW;

  // Issue of one product D (+)= A B over the staged K chunk kc (A holds time
  // columns [kc*KC, kc*KC + KC)) by the elected thread, and the bounded wait for
  // its completion (false if it never arrived).  Between the two, the block
  // issues the global loads of the next chunk, so they run under the MMAs.
  auto issue_mma = [&](uint32_t d, int kc) {
    proxy_fence();
    __syncthreads();
    if (tid == 0 && !no_commit) {
      tc_fence_after();
#pragma unroll 1
      for (int j = 0; j < KC / 8; ++j) {
        const int jb = kc * (KC / 8) + j;
        const uint64_t ah = tc_desc(a_hi + 2u * j * LBO_A, LBO_A, SBO);
        const uint64_t al = tc_desc(a_lo + 2u * j * LBO_A, LBO_A, SBO);
        const uint64_t bh = tc_desc(b_hi + 2u * jb * LBO_B, LBO_B, SBO);
        const uint64_t bl = tc_desc(b_lo + 2u * jb * LBO_B, LBO_B, SBO);
        tc_mma(d, ah, bh, IDESC, (kc > 0 || j > 0) ? 1u : 0u);
        tc_mma(d, ah, bl, IDESC, 1u);
        tc_mma(d, al, bh, IDESC, 1u);
      }
      tc_commit(mb);
    }
  };
  auto wait_mma = [&]() -> bool {
    const bool ok = mbar_wait(mb, parity, polls);
    parity ^= 1u;
    tc_fence_after();
    return __syncthreads_and(ok ? 1 : 0) != 0;
  };
  auto run_mma = [&](uint32_t d, int kc) -> bool {
    issue_mma(d, kc);
    return wait_mma();
  };

  // A operand chunks: K chunk kc (times [kc*KC, kc*KC + KC)) of the strip st's
  // modes, loaded into registers (consecutive threads: consecutive modes, so
  // every load instruction is coalesced), zero past the last mode or strip.
  constexpr int IT = TW * KC / 4 / kTcThreads;
  static_assert(IT * kTcThreads * 4 == TW * KC, "whole float4 groups per thread");
  auto load_chunk = [&](int st, int kc, float (&x)[IT][4]) {
    const int s0_ = st * TW;
    const bool live = st < nstrips;
#pragma unroll
    for (int u = 0; u < IT; ++u) {
      const int q = tid + u * kTcThreads;
      const int mm = q % TW, kq = q / TW;
      const int s = s0_ + mm;
      const int k0 = kc * KC + 4 * kq;
#pragma unroll
      for (int i = 0; i < 4; ++i) x[u][i] = (live && s < S) ? in[(long long)(k0 + i) * S + s] : 0.0f;
    }
  };
  auto stage_chunk = [&](const float (&x)[IT][4]) {
#pragma unroll
    for (int u = 0; u < IT; ++u) {
      const int q = tid + u * kTcThreads;
      const int mm = q % TW, kq = q / TW;
      float4 h, l;
      split4(x[u], h, l);
      const uint32_t off = kq * LBO_A + (mm >> 3) * 128u + (mm & 7) * 16u;
      *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Ahi) + off) = h;
      *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Alo) + off) = l;
    }
  };

  // The chunk to stage next, loaded one step ahead: during the previous chunk's
  // MMAs, or (the first chunk of the next strip) during the current strip's
  // division, second product and stores.
  float xr[IT][4];
  load_chunk(blockIdx.x, 0, xr);
  for (int strip = blockIdx.x; strip < nstrips; strip += gridDim.x) {
    const int s0 = strip * TW;
    const bool own = s0 + m < S;
    if (!failed) {
      for (int q = tid; q < TW; q += kTcThreads) {
        const int s = s0 + q;
        L1s[q] = s < S ? L1[s] : 1.0f;
        L2s[q] = s < S ? L2[s] : 0.0f;
      }
      // ---- product 1: D1[m][r] = sum_k X[k][s0 + m] V[r][k]
      for (int kc = 0; kc < NKC && !failed; ++kc) {
        stage_chunk(xr);
        issue_mma(d1, kc);
        if (kc + 1 < NKC)
          load_chunk(strip, kc + 1, xr);
        else
          load_chunk(strip + gridDim.x, 0, xr);
        failed = !wait_mma();
      }
    }
    if (!failed) {
      // ---- divide: this thread's mode m, times [half*NT/2, half*NT/2 + NT/2)
      float y[HALF];
#pragma unroll
      for (int c = 0; c < HALF; c += 16) {
        float v[16];
        tmem_ld16(d1 + lane_bits + (uint32_t)(half * HALF + c), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) y[c + i] = v[i];
      }
      const float l1 = L1s[m], l2 = L2s[m];
#pragma unroll
      for (int i = 0; i < HALF; ++i) y[i] = own ? y[i] / (l1 + lams[half * HALF + i] * l2) : 0.0f;
      tc_fence_before();
      // ---- product 2: D2[m][a] = sum_b Y[b][s0 + m] V[a][b]   (V^T = V)
      for (int kc = 0; kc < NKC && !failed; ++kc) {
        if (NKC == 1 || half == kc) {
#pragma unroll
          for (int i = 0; i < HALF; i += 4) {
            const int kl = half * HALF + i - kc * KC;  // time index within the staged chunk
            const float x[4] = {y[i], y[i + 1], y[i + 2], y[i + 3]};
            float4 h, l;
            split4(x, h, l);
            const uint32_t off = (uint32_t)(kl >> 2) * LBO_A + (m >> 3) * 128u + (m & 7) * 16u;
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Ahi) + off) = h;
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Alo) + off) = l;
          }
        }
        failed = !run_mma(d2, kc);
      }
    }
    if (!failed) {
      // ---- out[r][s0 + m] = D2[m][r]: coalesced along the spatial modes
#pragma unroll
      for (int c = 0; c < HALF; c += 16) {
        float v[16];
        tmem_ld16(d2 + lane_bits + (uint32_t)(half * HALF + c), v);
        if (own) {
#pragma unroll
          for (int i = 0; i < 16; ++i) out[(long long)(half * HALF + c + i) * S + s0 + m] = v[i];
        }
      }
      tc_fence_before();
      __syncthreads();  // accumulators read, L1s/L2s free before the next strip
      tc_fence_after();
    } else if (own) {
      // a completion never arrived: mark this strip's output as invalid
      for (int r = half * HALF; r < half * HALF + HALF; ++r) out[(long long)r * S + s0 + m] = __int_as_float(0x7fc00000);
    }
  }
  if (failed) {
    if (tid == 0 && sc != nullptr) {
      sc->status = MFG_ERR_TIMEOUT;
      sc->cg_done = 1;
    }
    mbar_wait(mb, parity ^ 1u, polls);  // let an MMA still in flight finish (bounded) before freeing its columns
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
  }
}

// Resident blocks per SM of each instantiation (set by time_tc_configure).
int g_tc_blocks_per_sm[3] = {1, 1, 1};

template <int NT>
void launch_tc(const float* in, float* out, const float* V, const float* lamt, const float* L1, const float* L2,
               int S, DevScalars* sc, cudaStream_t s) {
  const int nstrips = (S + kTcTW - 1) / kTcTW;
  const int per_sm = g_tc_blocks_per_sm[NT == 32 ? 0 : (NT == 64 ? 1 : 2)];
  const int cap = 152 * per_sm;  // one wave of resident blocks; each walks strips
  const int blocks = nstrips < cap ? nstrips : cap;
  k_time_tc<NT><<<blocks, kTcThreads, TcShape<NT>::smem, s>>>(in, out, V, lamt, L1, L2, S, sc);
}

}  // namespace

bool time_tc_supported(int nt) { return nt == 32 || nt == 64 || nt == 128; }

void launch_time_tc(const float* in, float* out, const float* V, const float* lamt, const float* L1,
                    const float* L2, int nt, int S, const DevScalars* sc, cudaStream_t s) {
  DevScalars* scw = const_cast<DevScalars*>(sc);
  if (nt == 32) launch_tc<32>(in, out, V, lamt, L1, L2, S, scw, s);
  else if (nt == 64) launch_tc<64>(in, out, V, lamt, L1, L2, S, scw, s);
  else launch_tc<128>(in, out, V, lamt, L1, L2, S, scw, s);
}

int time_tc_configure() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_time_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcShape<32>::smem) != cudaSuccess;
  bad |= cudaFuncSetAttribute(k_time_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcShape<64>::smem) != cudaSuccess;
  bad |= cudaFuncSetAttribute(k_time_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcShape<128>::smem) != cudaSuccess;
  // Resident blocks per SM from the kernel's own attributes: registers (in
  // their allocation unit of 8 per thread), shared memory (dynamic + static +
  // the 1 KB the driver reserves per block) and tensor-memory columns.  (The
  // occupancy API reported 1 block for the N_t = 32 kernel, whose registers
  // and shared memory admit 2 and 3; the blocks are independent, so a grid of
  // what fits is safe either way.)
  int dev = 0, smem_sm = 0, regs_sm = 0;
  bad |= cudaGetDevice(&dev) != cudaSuccess;
  bad |= cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess;
  bad |= cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess;
  const void* fns[3] = {(const void*)k_time_tc<32>, (const void*)k_time_tc<64>, (const void*)k_time_tc<128>};
  const size_t smem[3] = {TcShape<32>::smem, TcShape<64>::smem, TcShape<128>::smem};
  const int cols[3] = {64, 128, 256};
  for (int i = 0; i < 3; ++i) {
    cudaFuncAttributes fa{};
    bad |= cudaFuncGetAttributes(&fa, fns[i]) != cudaSuccess;
    const int regs = ((fa.numRegs + 7) / 8) * 8 * kTcThreads;
    int b = regs > 0 ? regs_sm / regs : 1;
    const int by_smem = (int)((size_t)smem_sm / (smem[i] + fa.sharedSizeBytes + 1024));
    if (by_smem < b) b = by_smem;
    if (b * cols[i] > 512) b = 512 / cols[i];
    g_tc_blocks_per_sm[i] = b < 1 ? 1 : b;
  }
  return bad ? MFG_ERR_CUDA : MFG_OK;
}

}  // namespace mfg
