// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "../../include/mfg.h"

namespace mfg {

constexpr int kThreads = 256;        // threads per block for 1-D launches
// Fixed grid of the grid-stride reduction kernels.  Kept small: every thread
// pays a warp-shuffle tree of FP64 adds at the end, and FP64 issue is scarce.
constexpr int kRedBlocks = 152 * 2;
constexpr int kVecBlocksMax = 152 * 4;   // largest vec_blocks the autotuner tries
constexpr int kAatWantDefault = 152 * 8;
constexpr int kAatWantMax = 152 * 16;    // largest aat_want the autotuner tries
constexpr int kMaxNt = 256;          // largest N_t of the fused time-transform kernel

// Geometry and coefficients of one instance on the device.  Internally every
// instance is a 2-axis grid: a 1-D problem is stored as Nx_int = 1 (inactive x
// axis) and Ny_int = N, so its two w planes are the y-axis components.
struct Geom {
  int nx, ny, nt;   // internal sizes
  int S;            // nx*ny
  long long n;      // nt*S
  int perx, pery;   // 1 = periodic axis, 0 = Neumann
  int actx;         // x axis carries terms (dim == 2)
  int c;            // primal planes: 3 or 5
  double ax, ay;    // 1/dx^2, 1/dy^2 (ax = 0 on an inactive axis)
  double idx, idy;  // 1/dx, 1/dy
  double idt;       // 1/dt
  double nu;
  // Launch choices: defaults from make_geom, replaced by mfg_autotune's
  // measured ones.  They change launch shapes and pass variants, never the
  // operator a kernel applies.
  int vec_blocks;   // grid cap of the vector and reduction kernels
  int aat_want;     // target block count of the AAt stencil launch
  int time_simt;    // 1: time pass on the CUDA cores even where the tensor-core pass applies
  int fft_x, fft_y; // 1: FFT spatial pass where the axis length allows it; 0: dense pass
  // Viscosity field (mfg_problem::nu_field): per node, the coefficient of its
  // "plus" face on each axis, nu_face * ax (kfx) and nu_face * ay (kfy), face i
  // joining nodes i and i+1 (wrapped on a periodic axis, 0 past a Neumann end);
  // the "minus" face of a node is the plus face of its minus neighbour.  Null
  // for a constant nu.  Device arrays of S doubles owned by the PrecTables.
  const double* kfx = nullptr;
  const double* kfy = nullptr;
};

// Coefficients of f_eff(m) = a m + b m^2 + c(x) (Sec. 2 calF).
struct Coef {
  double f_a, f_b, g_a;  // g enters the last plane divided by dt
  double gamma;
  double qprime;         // Hamiltonian exponent q' (eq. power_hamiltonian)
};

// Per-instance scalar state in device memory, written by the last block of the
// reduction kernels.  Keeping it on the device lets a whole solve run as one
// graph launch with no host round trip.
struct DevScalars {
  // Chambolle-Pock; theta = 1/sqrt(1 + 2 gamma tau) and 1/(2 tau) of the
  // current step, formed once per iteration for the prox kernel
  double tau, sigma, r_last, dm2;
  double theta, half_itau;
  double cg_tol;        // relative tolerance of the current solve
  double cp_tol;
  int ell, cp_left, cp_done, status;
  long long cg_total;
  int cg_max, cp_iters;
  // PCG
  double bnorm2, rz, pq, alpha, beta, rr, qz;
  int cg_it, cg_done, max_cg, cg_rule;
  double cg_tol_fixed;
  unsigned int counter;  // last-block ticket
  int inject;            // test hook (mfg_set_fault_injection); 0 in normal runs
};

// Host helpers (mfg_api.cu): problem validation (sets the error text),
// internal geometry, and the thread-local error record.
int validate_problem(const mfg_problem& p, int idx);
Geom make_geom(const mfg_problem& p);
int set_error(int code, const std::string& msg);

// Grid-stride 1-D launch shape shared by reduction kernels: enough blocks
// for one element per thread, at most `cap`.
inline int red_blocks(long long n, int cap = kRedBlocks) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// ---------------------------------------------------------------- kernels --
// Stencils (k_stencil.cu).
// Az (mode 1 only, MFG_CG_REF_RHS): AAt z_l on entry, b = AAt z_l + r on exit.
void launch_apply_C(const Geom& g, const double* v, double* r, double alpha, const double* m0,
                    double* partials, DevScalars* sc, int mode, cudaStream_t s,
                    const double* pdot = nullptr, double* Az = nullptr);
void launch_apply_Ct(const Geom& g, const double* p, double* x, cudaStream_t s);
// df64 != 0 selects the double-float variant of the stencil (MFG_MIXED_DF).
// q = AAt p.  scratch: 2 n doubles.  mode 0: plain apply; 1: PCG step (p.q, alpha).
void launch_AAt(const Geom& g, const double* p, double* q, double* scratch, double* partials,
                DevScalars* sc, int mode, cudaStream_t s, int df64);
int aat_kernel_count(int df64);
int aat_blocks(const Geom& g);

// Vector kernels (k_cg.cu).
// `cap`: grid cap (Geom::vec_blocks).
void launch_init_p(long long n, const double* zp, double* p, const double* r, double* partials,
                   DevScalars* sc, cudaStream_t s, int cap = kRedBlocks);
void launch_update_zr(long long n, double* z, double* r, const double* p, const double* q,
                      double* partials, DevScalars* sc, cudaStream_t s, int cap = kRedBlocks);
void launch_dot_beta(long long n, const double* r, const double* zp, const double* q, int flexible,
                     double* partials, DevScalars* sc, cudaStream_t s, int cap = kRedBlocks);
void launch_update_p(long long n, const double* zp, double* p, DevScalars* sc,
                     cudaGraphConditionalHandle h, int use_handle, cudaStream_t s, int cap = kRedBlocks);
void launch_scalars_begin(DevScalars* sc, cudaGraphConditionalHandle h, int use_handle,
                          cudaStream_t s);

// Preconditioner (k_precond.cu).  Tables are per instance, FP64 and FP32.
struct PrecTables {
  int nx, ny, nt;
  double *Hx64, *Hy64, *Vt64, *lamt64, *L1_64, *L2_64;  // device, FP64
  float *Hx32, *Hy32, *Vt32, *lamt32, *L1_32, *L2_32;   // device, FP32
  // FFT twiddles for power-of-two axes (null otherwise): tw (N/2 complex),
  // dct (N complex) per axis, both precisions.
  double *twx64 = nullptr, *dctx64 = nullptr, *twy64 = nullptr, *dcty64 = nullptr;
  float *twx32 = nullptr, *dctx32 = nullptr, *twy32 = nullptr, *dcty32 = nullptr;
  // l = 0 (exact time solve): Thomas factors c_k(s), 1/den_k(s) (n each) and
  // the off-diagonal per mode (S); null otherwise.
  double *thc64 = nullptr, *thd64 = nullptr, *tho64 = nullptr;
  float *thc32 = nullptr, *thd32 = nullptr, *tho32 = nullptr;
  // Viscosity field: face coefficients (Geom::kfx, kfy) and the banded Cholesky
  // factors of the per-frequency systems (k_band.cu); null otherwise.
  double *kfx = nullptr, *kfy = nullptr;
  int band_w = 0;                 // half-bandwidth w of the factors
  int* band_perm = nullptr;       // band position -> plane index (S ints)
  // Substitution stages of frequency k, forward (c) and backward (r): one
  // stage of G (w + G) values (rounded up to 16 bytes) per block of G steps,
  // at offset k nblk stage (layout in k_band.cu).  One precision is
  // allocated: FP64 for MFG_FP64, FP32 otherwise.
  double *bandc64 = nullptr, *bandr64 = nullptr;
  float *bandc32 = nullptr, *bandr32 = nullptr;
};
// Tensor-core time pass (MFG_MIXED_TC), for N_t in {32, 64, 128}.
bool time_tc_supported(int nt);
void launch_time_tc(const float* in, float* out, const float* V, const float* lamt, const float* L1,
                    const float* L2, int nt, int S, const DevScalars* sc, cudaStream_t s);
int time_tc_configure();
int build_prec_tables(const mfg_problem& p, const Geom& g, PrecTables* t, std::string* err);
void free_prec_tables(PrecTables* t);
// Operands of the PCG dot products that the last preconditioner pass can fuse
// (r.zp and, for the flexible variant, q.zp, then beta).
struct PcgDot {
  const double* r;
  const double* q;
  double* partials;
  DevScalars* sc;
  int flex;
};
// The PCG step z += alpha p, r -= alpha q (with its convergence test) that the
// first preconditioner pass can fuse.
struct PcgZr {
  double* z;
  double* r;
  const double* p;
  const double* q;
  double* partials;
  DevScalars* sc;
};
// z = P^{-1} r.  work64: 2n doubles (FP64 path); work32: 2n floats (mixed path).
// With zr != nullptr the PCG update of (z, r) runs first (fused into the first
// pass when it is an FFT pass, else by k_update_zr), and the transform is of
// the updated r; with dot != nullptr the PCG dot products and beta are formed
// afterwards (fused into the last FFT pass, else by k_dot_beta).
void launch_precond(const Geom& g, const PrecTables& t, int precision, const double* r, double* z,
                    double* work64, float* work32, const DevScalars* sc, cudaStream_t s,
                    const PcgDot* dot = nullptr, const PcgZr* zr = nullptr);
int precond_kernel_count(const Geom& g);
int precond_step_kernel_count(const Geom& g, const PrecTables& t);
// Viscosity field (k_band.cu): face coefficients and the banded factors of the
// per-frequency systems, built on the host in FP64 (lamt: the time
// eigenvalues); the preconditioner apply through them.
int build_band_tables(const mfg_problem& p, const Geom& g, const double* lamt, PrecTables* t,
                      std::string* err);
void launch_precond_band(const Geom& g, const PrecTables& t, int precision, const double* r, double* z,
                         double* work64, float* work32, const DevScalars* sc, cudaStream_t s);
int band_configure();
int precond_configure();

// FFT spatial passes (k_fft.cu).
bool fft_supported(int N);
long long fft_dot_partials(const Geom& g);
int fft_configure();
template <typename T>
void fft_y_forward(int N, int periodic, const double* in, T* out, const T* tw, const T* dct,
                   long long nlines, const DevScalars* sc, cudaStream_t s, const PcgZr* zr);
template <typename T>
void fft_y_inverse(int N, int periodic, const T* in, double* out, const T* tw, const T* dct,
                   long long nlines, const DevScalars* sc, cudaStream_t s, const PcgDot* dot);
template <typename T>
void fft_x(int N, int periodic, int inverse, const T* in, T* out, const T* tw, const T* dct,
           long long inner, long long outer, const DevScalars* sc, cudaStream_t s);

// Adjoint (k_adjoint.cu).
void launch_hinv(const Geom& g, const Coef& cf, const double* y, const double* u, double* out,
                 cudaStream_t s);
void launch_ct_hinv(const Geom& g, const Coef& cf, const double* y, const double* p,
                    const double* gsub, double* out, cudaStream_t s, const DevScalars* sc);
void launch_adj_grads(const Geom& g, const double* y, const double* z, const double* eta,
                      const double* mu, double* dm0, double* dV, double* dW, double* dnu,
                      double* partials, DevScalars* sc, cudaStream_t s);

// Prox (k_prox.cu).
// Az, rfin (MFG_CG_REF_RHS, else null): Az -= rfin turns the right-hand side b
// into AAt z_{l+1} = b - r_final for the next iteration's stop reference.
void launch_prox_cp(const Geom& g, const Coef& cf, const double* z, double* y, double* ybar,
                    const double* V, const double* W, double* partials, DevScalars* sc,
                    cudaGraphConditionalHandle h, int use_handle, cudaStream_t s,
                    double* Az = nullptr, const double* rfin = nullptr);
void launch_prox_plain(const Geom& g, const Coef& cf, double tau, const double* v, double* y,
                       const double* V, const double* W, cudaStream_t s);
int prox_configure();

}  // namespace mfg
