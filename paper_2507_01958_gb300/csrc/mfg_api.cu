// C ABI of the library (include/mfg.h): plan construction, the graph-captured
// Chambolle-Pock solve and the standalone operator entry points.
//
// mfg_solve runs the whole solve as ONE CUDA graph launch.  Per instance the
// graph holds a while-node over CP iterations (Sec. 3 eq. pasosChamPock) whose
// body is
//   r = sigma (C ybar - d)            k_apply_C (mode 1)
//   zp = P^{-1} r                     preconditioner passes (Alg. 1 + Alg. 2)
//   p = zp, rz = r.zp                 k_init_p
//   arm the inner while-node          k_scalars_begin
//   while (!converged): q = AAt p; z += alpha p, r -= alpha q; zp = P^{-1} r;
//                       beta; p = zp + beta p
//   prox + extrapolation + step sizes k_prox_cp (decides whether to loop again)
// Batched instances are independent branches of the same graph, so the
// runtime may overlap them on the GPU.  All control flow (convergence tests,
// step sizes) lives in device memory; the host only reads the final record.
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mfg_internal.cuh"

using namespace mfg;

namespace {
thread_local std::string g_last_error;
}  // namespace

int mfg::set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

namespace {

int fail(int code, const std::string& msg) { return mfg::set_error(code, msg); }

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(MFG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

struct Inst {
  mfg_problem p{};
  Geom g{};
  Coef cf{};
  PrecTables tabs{};
  size_t field_off = 0, primal_off = 0, dual_off = 0;
  double *r = nullptr, *pv = nullptr, *q = nullptr, *zp = nullptr, *work64 = nullptr;
  float* work32 = nullptr;
  double* partials = nullptr;
  DevScalars* sc = nullptr;  // points into the plan's contiguous array
  double *adj_t = nullptr, *adj_eta = nullptr;  // adjoint workspace, allocated on first use
  double* Az = nullptr;  // MFG_CG_REF_RHS: AAt z, carried across CP iterations (stop reference)
  int tuned = 0, measured = 0;                  // launch choices from mfg_autotune
  double tune_precond_us = 0.0, tune_aat_us = 0.0;
};

}  // namespace

namespace mfg {

int validate_problem(const mfg_problem& p, int idx) {
  const std::string at = " (instance " + std::to_string(idx) + ")";
  if (p.dim != 1 && p.dim != 2) return set_error(MFG_ERR_INVALID_ARG, "dim must be 1 or 2" + at);
  if (!(p.qprime >= 1.05 && p.qprime <= 20.0))
    return set_error(MFG_ERR_UNSUPPORTED, "the Hamiltonian exponent q' must lie in [1.05, 20]" + at);
  for (int a = 0; a < p.dim; ++a) {
    if (p.n[a] < 2) return set_error(MFG_ERR_INVALID_ARG, "grid sizes must be >= 2" + at);
    if (!(p.len[a] > 0.0)) return set_error(MFG_ERR_INVALID_ARG, "domain lengths must be > 0" + at);
    if (p.bc[a] != MFG_PERIODIC && p.bc[a] != MFG_NEUMANN)
      return set_error(MFG_ERR_INVALID_ARG, "bc must be MFG_PERIODIC or MFG_NEUMANN" + at);
  }
  if (p.nt < 2) return set_error(MFG_ERR_INVALID_ARG, "nt must be >= 2" + at);
  if (p.nt > kMaxNt) return set_error(MFG_ERR_UNSUPPORTED, "nt above 256 is not built" + at);
  if (!(p.T > 0.0)) return set_error(MFG_ERR_INVALID_ARG, "T must be > 0" + at);
  if (!(p.nu >= 0.0)) return set_error(MFG_ERR_INVALID_ARG, "nu must be >= 0" + at);
  if (!(p.f_a >= 0.0) || !(p.f_b >= 0.0) || !(p.g_a >= 0.0))
    return set_error(MFG_ERR_INVALID_ARG, "f_a, f_b, g_a must be >= 0 (monotone couplings)" + at);
  if (p.l != 0 && p.l != 1 && p.l != 2) return set_error(MFG_ERR_INVALID_ARG, "l must be 0, 1 or 2" + at);
  if (!(p.gamma > 0.0) || !(p.tau0 > 0.0) || !(p.sigma0 > 0.0))
    return set_error(MFG_ERR_INVALID_ARG, "gamma, tau0, sigma0 must be > 0" + at);
  if (p.max_cp < 0 || p.max_cg < 1) return set_error(MFG_ERR_INVALID_ARG, "max_cp >= 0, max_cg >= 1" + at);
  if (p.cg_rule != MFG_CG_FIXED && p.cg_rule != MFG_CG_ADAPTIVE)
    return set_error(MFG_ERR_INVALID_ARG, "cg_rule must be MFG_CG_FIXED or MFG_CG_ADAPTIVE" + at);
  if (p.cg_rule == MFG_CG_FIXED && !(p.cg_tol > 0.0))
    return set_error(MFG_ERR_INVALID_ARG, "cg_tol must be > 0" + at);
  if (p.cg_ref != MFG_CG_REF_RHS && p.cg_ref != MFG_CG_REF_RESID)
    return set_error(MFG_ERR_INVALID_ARG, "cg_ref must be MFG_CG_REF_RHS or MFG_CG_REF_RESID" + at);
  if (p.precision != MFG_FP64 && p.precision != MFG_MIXED && p.precision != MFG_MIXED_DF &&
      p.precision != MFG_MIXED_TC)
    return set_error(MFG_ERR_INVALID_ARG,
                     "precision must be MFG_FP64, MFG_MIXED, MFG_MIXED_DF or MFG_MIXED_TC" + at);
  const double nxy = (double)p.n[0] * (p.dim == 2 ? p.n[1] : 1);
  if (nxy * p.nt > 4.0e9) return set_error(MFG_ERR_INVALID_ARG, "instance too large" + at);
  if (p.nu_field != nullptr) {
    if (p.l == 0)
      return set_error(MFG_ERR_UNSUPPORTED, "a viscosity field needs l = 1 or 2 (the exact time solve is per Laplacian mode)" + at);
    const long long cnt = (long long)nxy;
    for (long long a = 0; a < cnt; ++a)
      if (!(p.nu_field[a] >= 0.0) || !std::isfinite(p.nu_field[a]))
        return set_error(MFG_ERR_INVALID_ARG, "viscosity field values must be finite and >= 0" + at);
  }
  return MFG_OK;
}

Geom make_geom(const mfg_problem& p) {
  Geom g{};
  g.nt = p.nt;
  g.nu = p.nu;
  g.idt = p.nt / p.T;
  auto spacing = [&](int a) { return p.len[a] / (p.bc[a] == MFG_PERIODIC ? p.n[a] : p.n[a] + 1); };
  if (p.dim == 1) {
    const double dx = spacing(0);
    g.nx = 1;
    g.ny = p.n[0];
    g.perx = 1;
    g.pery = p.bc[0] == MFG_PERIODIC;
    g.actx = 0;
    g.ax = 0.0;
    g.idx = 0.0;
    g.ay = 1.0 / (dx * dx);
    g.idy = 1.0 / dx;
    g.c = 3;
  } else {
    const double dx = spacing(0), dy = spacing(1);
    g.nx = p.n[0];
    g.ny = p.n[1];
    g.perx = p.bc[0] == MFG_PERIODIC;
    g.pery = p.bc[1] == MFG_PERIODIC;
    g.actx = 1;
    g.ax = 1.0 / (dx * dx);
    g.ay = 1.0 / (dy * dy);
    g.idx = 1.0 / dx;
    g.idy = 1.0 / dy;
    g.c = 5;
  }
  g.S = g.nx * g.ny;
  g.n = (long long)g.S * g.nt;
  g.vec_blocks = kRedBlocks;
  g.aat_want = kAatWantDefault;
  g.time_simt = 0;
  g.fft_x = g.fft_y = 1;
  return g;
}

}  // namespace mfg

struct mfg_plan_s {
  int device = 0;
  std::vector<Inst> inst;
  size_t field_total = 0, primal_total = 0, dual_total = 0;
  DevScalars* sc_dev = nullptr;
  DevScalars* sc_host = nullptr;  // pinned
  long long launches = 0;
  // graph cache
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaStream_t cap0 = nullptr, cap1 = nullptr;
  int launch_mode = MFG_LAUNCH_GRAPH;
  int inject = MFG_INJECT_NONE;  // test hook, copied into the device scalars by mfg_solve
  // device staging for mfg_solve_host
  double *h_m0 = nullptr, *h_V = nullptr, *h_W = nullptr, *h_y = nullptr, *h_ybar = nullptr,
         *h_z = nullptr;
};

namespace {

void free_inst(Inst& in) {
  free_prec_tables(&in.tabs);
  void* ptrs[] = {in.r, in.pv, in.q, in.zp, in.work64, in.work32, in.partials, in.adj_t, in.adj_eta, in.Az};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  in.r = in.pv = in.q = in.zp = in.work64 = in.partials = in.adj_t = in.adj_eta = in.Az = nullptr;
  in.work32 = nullptr;
}

void drop_graph(mfg_plan_t pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->exec = nullptr;
  pl->graph = nullptr;
  for (auto& k : pl->key) k = nullptr;
}

int check_b(mfg_plan_t pl, int b) {
  if (!pl) return fail(MFG_ERR_INVALID_ARG, "null plan");
  if (b < 0 || b >= (int)pl->inst.size()) return fail(MFG_ERR_INVALID_ARG, "instance index out of range");
  return MFG_OK;
}

// kernels per CP iteration outside PCG (rhs, precond, init_p, arm, prox), per
// PCG iteration, and once per solve (the AAt z of the MFG_CG_REF_RHS reference)
int launches_cp(const Inst& in) { return 4 + precond_kernel_count(in.g); }
int launches_solve(const Inst& in) { return in.Az ? aat_kernel_count(in.p.precision == MFG_MIXED_DF) : 0; }

// Stop reference of MFG_CG_REF_RHS, ||b|| of the system of eq. CC*: the
// right-hand side b = AAt z_l + sigma (C ybar - d) needs AAt z_l.  It is
// applied once per solve to the caller's z; afterwards the CP loop carries it:
// the rhs kernel turns Az into b, the prox kernel subtracts the final PCG
// residual (AAt z_{l+1} = b - r_final, up to the recursive residual's
// rounding).
void launch_stop_reference_start(const Inst& in, const double* z, cudaStream_t s) {
  if (!in.Az) return;
  launch_AAt(in.g, z, in.Az, in.work64, in.partials, in.sc, 0, s, in.p.precision == MFG_MIXED_DF);
}
int launches_cg(const Inst& in) {
  return 1 + aat_kernel_count(in.p.precision == MFG_MIXED_DF) + precond_step_kernel_count(in.g, in.tabs);
}

// Captures the per-instance CP loop into `top` as a while-node branch.
int add_instance(mfg_plan_t pl, Inst& in, cudaGraph_t top, const double* m0, const double* V,
                 const double* W, double* y, double* ybar, double* z) {
  // prologue: AAt z of the stop reference, before the CP loop
  std::vector<cudaGraphNode_t> pro;
  if (in.Az) {
    cudaStream_t s0 = pl->cap0;
    CK(cudaStreamBeginCaptureToGraph(s0, top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_stop_reference_start(in, z, s0);
    cudaStreamCaptureStatus cst0;
    const cudaGraphNode_t* d0 = nullptr;
    size_t n0 = 0;
    CK(cudaStreamGetCaptureInfo(s0, &cst0, nullptr, nullptr, &d0, nullptr, &n0));
    pro.assign(d0, d0 + n0);
    cudaGraph_t tg = top;
    CK(cudaStreamEndCapture(s0, &tg));
  }
  cudaGraphConditionalHandle hc, hg;
  CK(cudaGraphConditionalHandleCreate(&hc, top, in.p.max_cp > 0 ? 1u : 0u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wcp;
  CK(cudaGraphAddNode(&wcp, top, pro.empty() ? nullptr : pro.data(), nullptr, pro.size(), &cp));
  cudaGraph_t body_cp = cp.conditional.phGraph_out[0];
  CK(cudaGraphConditionalHandleCreate(&hg, body_cp, 0, 0));

  const Geom& g = in.g;
  const int flex = in.p.precision != MFG_FP64;
  const int dfa = in.p.precision == MFG_MIXED_DF;
  cudaStream_t s = pl->cap0;
  CK(cudaStreamBeginCaptureToGraph(s, body_cp, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_apply_C(g, ybar, in.r, 1.0, m0, in.partials, in.sc, 1, s, nullptr, in.Az);
  launch_precond(g, in.tabs, in.p.precision, in.r, in.zp, in.work64, in.work32, in.sc, s);
  launch_init_p(g.n, in.zp, in.pv, in.r, in.partials, in.sc, s, g.vec_blocks);
  launch_scalars_begin(in.sc, hg, 1, s);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  cudaGraphNodeParams cg{};
  cg.type = cudaGraphNodeTypeConditional;
  cg.conditional.handle = hg;
  cg.conditional.type = cudaGraphCondTypeWhile;
  cg.conditional.size = 1;
  cudaGraphNode_t wcg;
  CK(cudaGraphAddNode(&wcg, body_cp, deps, nullptr, ndeps, &cg));
  cudaGraph_t body_cg = cg.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(s, &wcg, nullptr, 1, cudaStreamSetCaptureDependencies));
  launch_prox_cp(g, in.cf, z, y, ybar, V, W, in.partials, in.sc, hc, 1, s, in.Az, in.r);
  CK(cudaStreamEndCapture(s, &body_cp));

  cudaStream_t s2 = pl->cap1;
  CK(cudaStreamBeginCaptureToGraph(s2, body_cg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const PcgDot dot{in.r, in.q, in.partials, in.sc, flex};
  const PcgZr zr{z, in.r, in.pv, in.q, in.partials, in.sc};
  launch_AAt(g, in.pv, in.q, in.work64, in.partials, in.sc, 1, s2, dfa);
  launch_precond(g, in.tabs, in.p.precision, in.r, in.zp, in.work64, in.work32, in.sc, s2, &dot, &zr);
  launch_update_p(g.n, in.zp, in.pv, in.sc, hg, 1, s2, g.vec_blocks);
  CK(cudaStreamEndCapture(s2, &body_cg));
  return MFG_OK;
}

int build_graph(mfg_plan_t pl, const double* m0, const double* V, const double* W, double* y,
                double* ybar, double* z) {
  drop_graph(pl);
  CK(cudaGraphCreate(&pl->graph, 0));
  for (auto& in : pl->inst) {
    int rc = add_instance(pl, in, pl->graph, m0 + in.field_off, V + in.field_off, W + in.field_off,
                          y + in.primal_off, ybar + in.primal_off, z + in.dual_off);
    if (rc != MFG_OK) {
      drop_graph(pl);
      return rc;
    }
  }
  cudaError_t e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
  if (e != cudaSuccess) {
    drop_graph(pl);
    return fail(MFG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  const void* k[6] = {m0, V, W, y, ybar, z};
  for (int i = 0; i < 6; ++i) pl->key[i] = k[i];
  return MFG_OK;
}

// Kernel-by-kernel launch of the same solve on the caller's stream, with the
// host reading the convergence flags after every PCG iteration.  Same kernels
// and launch shapes as the graph; used for per-kernel profiling.
int solve_eager(mfg_plan_t pl, const double* m0, const double* V, const double* W, double* y,
                double* ybar, double* z, cudaStream_t s) {
  DevScalars hs;
  for (auto& in : pl->inst) {
    const Geom& g = in.g;
    const int flex = in.p.precision != MFG_FP64;
  const int dfa = in.p.precision == MFG_MIXED_DF;
    const double* m0b = m0 + in.field_off;
    const double* Vb = V + in.field_off;
    const double* Wb = W + in.field_off;
    double* yb = y + in.primal_off;
    double* ybb = ybar + in.primal_off;
    double* zb = z + in.dual_off;
    if (in.p.max_cp > 0) {
      launch_stop_reference_start(in, zb, s);
      pl->launches += launches_solve(in);
    }
    for (int it = 0; it < in.p.max_cp; ++it) {
      launch_apply_C(g, ybb, in.r, 1.0, m0b, in.partials, in.sc, 1, s, nullptr, in.Az);
      launch_precond(g, in.tabs, in.p.precision, in.r, in.zp, in.work64, in.work32, in.sc, s);
      launch_init_p(g.n, in.zp, in.pv, in.r, in.partials, in.sc, s, g.vec_blocks);
      pl->launches += launches_cp(in) - 2;  // the prox is counted below; nothing arms a graph node
      for (;;) {
        CK(cudaMemcpyAsync(&hs, in.sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hs.cg_done) break;
        const PcgDot dot{in.r, in.q, in.partials, in.sc, flex};
        const PcgZr zr{zb, in.r, in.pv, in.q, in.partials, in.sc};
        launch_AAt(g, in.pv, in.q, in.work64, in.partials, in.sc, 1, s, dfa);
        launch_precond(g, in.tabs, in.p.precision, in.r, in.zp, in.work64, in.work32, in.sc, s, &dot, &zr);
        launch_update_p(g.n, in.zp, in.pv, in.sc, 0, 0, s, g.vec_blocks);
        pl->launches += launches_cg(in);
      }
      launch_prox_cp(g, in.cf, zb, yb, ybb, Vb, Wb, in.partials, in.sc, 0, 0, s, in.Az, in.r);
      pl->launches += 1;
      CK(cudaMemcpyAsync(&hs, in.sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hs.cp_done || hs.cp_left <= 0) break;
    }
  }
  return MFG_OK;
}

// ------------------------------------------------------------- autotuner --
// Launch choices per instance shape (grid, N_t, boundary conditions,
// precision, time solve, viscosity field or not), measured once per process: a later plan with the
// same shape takes the cached choice without timing again.
using TuneKey = std::array<int, 9>;
struct TuneVal {
  int vec_blocks, aat_want, time_simt, fft_x, fft_y;
  double precond_us, aat_us;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

TuneKey tune_key(const Inst& in) {
  return TuneKey{in.g.nx, in.g.ny, in.g.nt, in.g.perx, in.g.pery, in.p.precision, in.p.l == 0 ? 1 : 0,
                 in.g.actx, in.g.kfy != nullptr ? 1 : 0};
}

// Fills a device buffer with a positive, finite pattern (bytes 0x3F), so that
// timed reductions see nonzero, well-scaled data.
int fill_pattern(void* p, size_t bytes, cudaStream_t s) {
  return cudaMemsetAsync(p, 0x3F, bytes, s) == cudaSuccess ? MFG_OK : MFG_ERR_CUDA;
}

// PCG scalars under which every timed kernel runs its full body: nothing
// converged, alpha = 0 (the fused z, r update leaves them unchanged).
int reset_tune_scalars(const Inst& in, cudaStream_t s) {
  DevScalars h{};
  h.status = MFG_OK;
  h.rz = 1.0;
  h.bnorm2 = 1.0;
  h.cg_tol = 0.0;
  h.max_cg = INT_MAX;
  return cudaMemcpyAsync(in.sc, &h, sizeof(h), cudaMemcpyHostToDevice, s) == cudaSuccess ? MFG_OK : MFG_ERR_CUDA;
}

// Mean time in microseconds of `f` on stream s (one warm-up call, then enough
// repetitions for about 2 ms, between 3 and 50).
template <typename F>
double time_us(F&& f, cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
  f();
  cudaEventRecord(a, s);
  f();
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  const double t0 = 1e3 * ms;
  int reps = t0 > 0 ? (int)std::ceil(2000.0 / t0) : 50;
  reps = reps < 3 ? 3 : (reps > 50 ? 50 : reps);
  cudaEventRecord(a, s);
  for (int i = 0; i < reps; ++i) f();
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b);
  return 1e3 * ms / reps;
}

// Times the candidates for one instance and keeps the fastest in in.g:
//   vector and reduction grid cap    152, 304, 608 blocks
//   preconditioner passes            time pass on the tensor cores or the CUDA
//                                    cores (MFG_MIXED_TC); FFT or dense pass per
//                                    power-of-two axis; timed as the PCG step
//                                    (fused z, r update and dot products)
//   AAt stencil target blocks        152 x 4, 8, 16
int tune_instance(Inst& in, double* zbuf, cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
  const long long n = in.g.n;
  int rc;
  if ((rc = fill_pattern(in.r, n * 8, s)) || (rc = fill_pattern(in.pv, n * 8, s)) ||
      (rc = fill_pattern(in.q, n * 8, s)) || (rc = fill_pattern(in.zp, n * 8, s)) ||
      (rc = fill_pattern(zbuf, n * 8, s)))
    return rc;
  const int flex = in.p.precision != MFG_FP64;
  Geom g = in.g;
  // vector kernels
  {
    double best = 1e300;
    int choice = g.vec_blocks;
    for (int cap : {152, 304, 608}) {
      g.vec_blocks = cap;
      if ((rc = reset_tune_scalars(in, s))) return rc;
      const double t = time_us([&] {
        launch_update_p(n, in.zp, in.pv, in.sc, 0, 0, s, cap);
        launch_init_p(n, in.zp, in.pv, in.r, in.partials, in.sc, s, cap);
      }, s, a, b);
      if (t < best) { best = t; choice = cap; }
    }
    g.vec_blocks = choice;
  }
  // preconditioner passes
  {
    const bool tc_opt = in.p.precision == MFG_MIXED_TC && time_tc_supported(g.nt) && in.p.l != 0;
    const bool fy_opt = fft_supported(g.ny) && in.tabs.twy32 != nullptr;
    const bool fx_opt = g.nx > 1 && fft_supported(g.nx) && in.tabs.twx32 != nullptr;
    double best = 1e300;
    Geom pick = g;
    for (int ts = 0; ts <= (tc_opt ? 1 : 0); ++ts)
      for (int fy = fy_opt ? 1 : 0; fy >= 0; --fy)
        for (int fx = fx_opt ? 1 : 0; fx >= 0; --fx) {
          Geom c = g;
          c.time_simt = tc_opt ? ts : 0;
          c.fft_y = fy;
          c.fft_x = fx;
          const PcgDot dot{in.r, in.q, in.partials, in.sc, flex};
          const PcgZr zr{zbuf, in.r, in.pv, in.q, in.partials, in.sc};
          if ((rc = reset_tune_scalars(in, s))) return rc;
          const double t = time_us([&] {
            launch_precond(c, in.tabs, in.p.precision, in.r, in.zp, in.work64, in.work32, in.sc, s, &dot, &zr);
          }, s, a, b);
          if (t < best) { best = t; pick = c; }
        }
    g = pick;
    in.tune_precond_us = best;
  }
  // AAt stencil chunking
  {
    double best = 1e300;
    int choice = g.aat_want;
    for (int want : {152 * 4, 152 * 8, 152 * 16}) {
      Geom c = g;
      c.aat_want = want;
      if ((rc = reset_tune_scalars(in, s))) return rc;
      const double t = time_us([&] {
        launch_AAt(c, in.pv, in.q, in.work64, in.partials, in.sc, 1, s, in.p.precision == MFG_MIXED_DF);
      }, s, a, b);
      if (t < best) { best = t; choice = want; }
    }
    g.aat_want = choice;
    in.tune_aat_us = best;
  }
  if (cudaGetLastError() != cudaSuccess) return fail(MFG_ERR_CUDA, "a launch failed while autotuning");
  in.g = g;
  in.measured = 1;
  in.tuned = 1;
  return MFG_OK;
}

}  // namespace

extern "C" {

int mfg_autotune(mfg_plan_t pl, void* stream) {
  if (!pl) return fail(MFG_ERR_INVALID_ARG, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  size_t nmax = 0;
  for (auto& in : pl->inst) nmax = std::max(nmax, (size_t)in.g.n);
  double* zbuf = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&zbuf, nmax * 8) != cudaSuccess) return fail(MFG_ERR_CUDA, "cudaMalloc failed for autotuning");
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaFree(zbuf);
    return fail(MFG_ERR_CUDA, "cudaEventCreate failed");
  }
  int rc = MFG_OK;
  for (auto& in : pl->inst) {
    const TuneKey key = tune_key(in);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        const TuneVal& v = it->second;
        in.g.vec_blocks = v.vec_blocks;
        in.g.aat_want = v.aat_want;
        in.g.time_simt = v.time_simt;
        in.g.fft_x = v.fft_x;
        in.g.fft_y = v.fft_y;
        in.tune_precond_us = v.precond_us;
        in.tune_aat_us = v.aat_us;
        in.tuned = 1;
        in.measured = 0;
        continue;
      }
    }
    rc = tune_instance(in, zbuf, s, a, b);
    if (rc != MFG_OK) break;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = TuneVal{in.g.vec_blocks, in.g.aat_want, in.g.time_simt, in.g.fft_x, in.g.fft_y,
                                in.tune_precond_us, in.tune_aat_us};
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(zbuf);
  drop_graph(pl);  // the next mfg_solve captures the new launch shapes
  if (rc != MFG_OK) return rc;
  CK(cudaGetLastError());
  return MFG_OK;
}

int mfg_get_schedule(mfg_plan_t pl, int b, mfg_schedule* out) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!out) return fail(MFG_ERR_INVALID_ARG, "null output");
  const Inst& in = pl->inst[b];
  const Geom& g = in.g;
  std::memset(out, 0, sizeof(*out));
  out->tuned = in.tuned;
  out->measured = in.measured;
  const bool tc = in.p.precision == MFG_MIXED_TC && time_tc_supported(g.nt) && in.p.l != 0 && !g.time_simt;
  out->time_pass = tc ? MFG_TIME_TENSOR_CORES : MFG_TIME_CUDA_CORES;
  const int fy = g.fft_y && fft_supported(g.ny) && in.tabs.twy32 != nullptr;
  const int fx = g.fft_x && g.nx > 1 && fft_supported(g.nx) && in.tabs.twx32 != nullptr;
  if (in.p.dim == 1) {
    out->fft[0] = fy;
  } else {
    out->fft[0] = fx;
    out->fft[1] = fy;
  }
  out->aat_blocks = aat_blocks(g);
  out->vec_blocks = g.vec_blocks;
  out->precond_us = in.tune_precond_us;
  out->aat_us = in.tune_aat_us;
  return MFG_OK;
}


int mfg_set_fault_injection(mfg_plan_t pl, int what) {
  if (!pl) return fail(MFG_ERR_INVALID_ARG, "null plan");
  if (what != MFG_INJECT_NONE && what != MFG_INJECT_TC_NO_COMMIT && what != MFG_INJECT_BAND_NO_COPY)
    return fail(MFG_ERR_INVALID_ARG,
                "what must be MFG_INJECT_NONE, MFG_INJECT_TC_NO_COMMIT or MFG_INJECT_BAND_NO_COPY");
  pl->inject = what;
  return MFG_OK;
}

int mfg_set_launch_mode(mfg_plan_t pl, int mode) {
  if (!pl) return fail(MFG_ERR_INVALID_ARG, "null plan");
  if (mode != MFG_LAUNCH_GRAPH && mode != MFG_LAUNCH_EAGER)
    return fail(MFG_ERR_INVALID_ARG, "mode must be MFG_LAUNCH_GRAPH or MFG_LAUNCH_EAGER");
  pl->launch_mode = mode;
  return MFG_OK;
}

const char* mfg_last_error(void) { return g_last_error.c_str(); }

int mfg_plan(const mfg_problem* probs, int batch, mfg_plan_t* out) {
  if (!out) return fail(MFG_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (!probs || batch < 1) return fail(MFG_ERR_INVALID_ARG, "need at least one problem");
  for (int b = 0; b < batch; ++b) {
    int rc = validate_problem(probs[b], b);
    if (rc != MFG_OK) return rc;
  }
  g_last_error.clear();
  auto* pl = new mfg_plan_s();
  CK(cudaGetDevice(&pl->device));
  if (precond_configure() != MFG_OK) {
    delete pl;
    return fail(MFG_ERR_CUDA, "cudaFuncSetAttribute failed");
  }
  pl->inst.resize(batch);
  size_t fo = 0, po = 0, dof = 0;
  auto bail = [&](int code, const std::string& msg) {
    mfg_destroy(pl);
    return fail(code, msg);
  };
  for (int b = 0; b < batch; ++b) {
    Inst& in = pl->inst[b];
    in.p = probs[b];
    in.g = make_geom(in.p);
    in.cf = Coef{in.p.f_a, in.p.f_b, in.p.g_a, in.p.gamma, in.p.qprime};
    in.field_off = fo;
    in.primal_off = po;
    in.dual_off = dof;
    fo += (size_t)in.g.S;
    po += (size_t)in.g.c * in.g.n;
    dof += (size_t)in.g.n;
    std::string err;
    int rc = build_prec_tables(in.p, in.g, &in.tabs, &err);
    if (rc != MFG_OK) return bail(rc, err);
    // a viscosity field lives on in the plan's face coefficients and factors;
    // the caller's array is not retained
    in.g.kfx = in.tabs.kfx;
    in.g.kfy = in.tabs.kfy;
    in.p.nu_field = nullptr;
    const size_t n = (size_t)in.g.n;
    // partial sums for the largest grids any launch choice may use
    Geom gmax = in.g;
    gmax.aat_want = kAatWantMax;
    size_t npart = (size_t)std::max<long long>(std::max(2 * kVecBlocksMax, aat_blocks(gmax)),
                                               fft_dot_partials(in.g));
    if (cudaMalloc(&in.r, n * 8) != cudaSuccess || cudaMalloc(&in.pv, n * 8) != cudaSuccess ||
        cudaMalloc(&in.q, n * 8) != cudaSuccess || cudaMalloc(&in.zp, n * 8) != cudaSuccess ||
        cudaMalloc(&in.partials, npart * 8) != cudaSuccess)
      return bail(MFG_ERR_CUDA, "cudaMalloc failed for solver workspace");
    if (in.p.precision != MFG_FP64) {
      if (cudaMalloc(&in.work32, 2 * n * 4) != cudaSuccess)
        return bail(MFG_ERR_CUDA, "cudaMalloc failed for FP32 workspace");
    }
    if (cudaMalloc(&in.work64, 2 * n * 8) != cudaSuccess)
      return bail(MFG_ERR_CUDA, "cudaMalloc failed for FP64 workspace");
    if (in.p.cg_ref == MFG_CG_REF_RHS && cudaMalloc(&in.Az, n * 8) != cudaSuccess)
      return bail(MFG_ERR_CUDA, "cudaMalloc failed for the stop-reference vector");
  }
  pl->field_total = fo;
  pl->primal_total = po;
  pl->dual_total = dof;
  if (cudaMalloc(&pl->sc_dev, sizeof(DevScalars) * batch) != cudaSuccess ||
      cudaMallocHost(&pl->sc_host, sizeof(DevScalars) * batch) != cudaSuccess)
    return bail(MFG_ERR_CUDA, "cudaMalloc failed for device scalars");
  std::memset(pl->sc_host, 0, sizeof(DevScalars) * batch);
  for (int b = 0; b < batch; ++b) pl->inst[b].sc = pl->sc_dev + b;
  if (cudaStreamCreateWithFlags(&pl->cap0, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&pl->cap1, cudaStreamNonBlocking) != cudaSuccess)
    return bail(MFG_ERR_CUDA, "cudaStreamCreate failed");
  *out = pl;
  return MFG_OK;
}

int mfg_destroy(mfg_plan_t pl) {
  if (!pl) return MFG_OK;
  drop_graph(pl);
  for (auto& in : pl->inst) free_inst(in);
  if (pl->sc_dev) cudaFree(pl->sc_dev);
  if (pl->sc_host) cudaFreeHost(pl->sc_host);
  double* hs[] = {pl->h_m0, pl->h_V, pl->h_W, pl->h_y, pl->h_ybar, pl->h_z};
  for (double* q : hs)
    if (q) cudaFree(q);
  if (pl->cap0) cudaStreamDestroy(pl->cap0);
  if (pl->cap1) cudaStreamDestroy(pl->cap1);
  delete pl;
  return MFG_OK;
}

int mfg_layout(mfg_plan_t pl, int b, size_t* field_off, size_t* primal_off, size_t* dual_off,
               size_t* n, int* c) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  const Inst& in = pl->inst[b];
  if (field_off) *field_off = in.field_off;
  if (primal_off) *primal_off = in.primal_off;
  if (dual_off) *dual_off = in.dual_off;
  if (n) *n = (size_t)in.g.n;
  if (c) *c = in.g.c;
  return MFG_OK;
}

int mfg_sizes(mfg_plan_t pl, size_t* field_total, size_t* primal_total, size_t* dual_total) {
  if (!pl) return fail(MFG_ERR_INVALID_ARG, "null plan");
  if (field_total) *field_total = pl->field_total;
  if (primal_total) *primal_total = pl->primal_total;
  if (dual_total) *dual_total = pl->dual_total;
  return MFG_OK;
}

long long mfg_kernel_launches(mfg_plan_t pl) { return pl ? pl->launches : -1; }

int mfg_solve(mfg_plan_t pl, const double* m0, const double* V, const double* W, double* y,
              double* ybar, double* z, mfg_stats* st, void* stream) {
  if (!pl) return fail(MFG_ERR_INVALID_ARG, "null plan");
  if (!m0 || !V || !W || !y || !ybar || !z || !st)
    return fail(MFG_ERR_INVALID_ARG, "null array or stats pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const int B = (int)pl->inst.size();
  for (int b = 0; b < B; ++b) {
    const Inst& in = pl->inst[b];
    DevScalars& h = pl->sc_host[b];
    std::memset(&h, 0, sizeof(h));
    const bool fresh = st[b].ell <= 0;
    h.tau = fresh ? in.p.tau0 : st[b].tau;
    h.sigma = fresh ? in.p.sigma0 : st[b].sigma;
    h.theta = 1.0 / std::sqrt(1.0 + 2.0 * in.p.gamma * h.tau);
    h.half_itau = 0.5 / h.tau;
    h.ell = fresh ? 0 : st[b].ell;
    h.r_last = fresh ? INFINITY : st[b].r_last;
    h.cp_tol = in.p.cp_tol;
    h.cp_left = in.p.max_cp;
    h.cp_done = in.p.max_cp <= 0;
    h.status = MFG_OK;
    h.max_cg = in.p.max_cg;
    h.cg_rule = in.p.cg_rule;
    h.cg_tol_fixed = in.p.cg_tol;
    h.inject = pl->inject;
  }
  const bool eager = pl->launch_mode == MFG_LAUNCH_EAGER;
  if (!eager) {
    const void* k[6] = {m0, V, W, y, ybar, z};
    bool same = pl->exec != nullptr;
    for (int i = 0; i < 6 && same; ++i) same = (pl->key[i] == k[i]);
    if (!same) {
      int rc = build_graph(pl, m0, V, W, y, ybar, z);
      if (rc != MFG_OK) return rc;
    }
  }
  CK(cudaMemcpyAsync(pl->sc_dev, pl->sc_host, sizeof(DevScalars) * B, cudaMemcpyHostToDevice, s));
  bool any = false;
  for (int b = 0; b < B; ++b) any = any || (pl->inst[b].p.max_cp > 0);
  if (any && eager) {
    int rc = solve_eager(pl, m0, V, W, y, ybar, z, s);
    if (rc != MFG_OK) return rc;
  } else if (any) {
    CK(cudaGraphLaunch(pl->exec, s));
  }
  CK(cudaMemcpyAsync(pl->sc_host, pl->sc_dev, sizeof(DevScalars) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  int first = MFG_OK;
  for (int b = 0; b < B; ++b) {
    const DevScalars& h = pl->sc_host[b];
    st[b].status = h.status;
    st[b].ell = h.ell;
    st[b].cp_iters = h.cp_iters;
    st[b].cg_iters = h.cg_total;
    st[b].max_cg_in_solve = h.cg_max;
    st[b].r_last = h.r_last;
    st[b].tau = h.tau;
    st[b].sigma = h.sigma;
    if (!eager)
      pl->launches += (long long)launches_cp(pl->inst[b]) * h.cp_iters + (long long)launches_cg(pl->inst[b]) * h.cg_total +
                      (pl->inst[b].p.max_cp > 0 ? launches_solve(pl->inst[b]) : 0);
    if (first == MFG_OK && h.status != MFG_OK) first = h.status;
  }
  if (first != MFG_OK) return fail(first, "an instance finished with a non-OK status");
  return MFG_OK;
}

int mfg_solve_host(mfg_plan_t pl, const double* m0, const double* V, const double* W, double* y,
                   double* ybar, double* z, mfg_stats* st, void* stream) {
  if (!pl) return fail(MFG_ERR_INVALID_ARG, "null plan");
  if (!m0 || !V || !W || !y || !ybar || !z || !st)
    return fail(MFG_ERR_INVALID_ARG, "null array or stats pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t F = pl->field_total * 8, P = pl->primal_total * 8, D = pl->dual_total * 8;
  if (!pl->h_m0) {
    if (cudaMalloc(&pl->h_m0, F) != cudaSuccess || cudaMalloc(&pl->h_V, F) != cudaSuccess ||
        cudaMalloc(&pl->h_W, F) != cudaSuccess || cudaMalloc(&pl->h_y, P) != cudaSuccess ||
        cudaMalloc(&pl->h_ybar, P) != cudaSuccess || cudaMalloc(&pl->h_z, D) != cudaSuccess)
      return fail(MFG_ERR_CUDA, "cudaMalloc failed for host-call staging buffers");
  }
  CK(cudaMemcpyAsync(pl->h_m0, m0, F, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pl->h_V, V, F, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pl->h_W, W, F, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pl->h_y, y, P, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pl->h_ybar, ybar, P, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pl->h_z, z, D, cudaMemcpyHostToDevice, s));
  int rc = mfg_solve(pl, pl->h_m0, pl->h_V, pl->h_W, pl->h_y, pl->h_ybar, pl->h_z, st, stream);
  if (rc != MFG_OK && rc != MFG_ERR_NOT_CONVERGED && rc != MFG_ERR_NONFINITE && rc != MFG_ERR_TIMEOUT)
    return rc;
  CK(cudaMemcpyAsync(y, pl->h_y, P, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ybar, pl->h_ybar, P, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(z, pl->h_z, D, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return rc;
}

int mfg_adjoint(mfg_plan_t pl, int b, const double* y, const double* z, const double* gy, double* dm0,
                double* dV, double* dW, double* dnu, double tol, int max_iter, mfg_stats* st,
                void* stream) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!y || !z || !gy || !dm0 || !dV || !dnu || !st)
    return fail(MFG_ERR_INVALID_ARG, "null array or stats pointer");
  if (!(tol > 0.0) || max_iter < 1) return fail(MFG_ERR_INVALID_ARG, "tol > 0 and max_iter >= 1 required");
  Inst& in = pl->inst[b];
  if (in.p.qprime != 2.0)
    return fail(MFG_ERR_UNSUPPORTED, "the adjoint is built for the quadratic Hamiltonian (q' = 2) only");
  const Geom& g = in.g;
  const size_t n = (size_t)g.n;
  if (!in.adj_t) {
    if (cudaMalloc(&in.adj_t, (size_t)g.c * n * 8) != cudaSuccess || cudaMalloc(&in.adj_eta, n * 8) != cudaSuccess)
      return fail(MFG_ERR_CUDA, "cudaMalloc failed for adjoint workspace");
  }
  cudaStream_t s = (cudaStream_t)stream;
  DevScalars h{};
  h.status = MFG_OK;
  h.cg_rule = MFG_CG_FIXED;
  h.cg_tol_fixed = tol;
  h.max_cg = max_iter;
  CK(cudaMemcpyAsync(in.sc, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  const int flex = in.p.precision != MFG_FP64;
  const int dfa = in.p.precision == MFG_MIXED_DF;
  // right-hand side C H^{-1} g; eta starts at 0
  launch_hinv(g, in.cf, y, gy, in.adj_t, s);
  launch_apply_C(g, in.adj_t, in.r, 1.0, nullptr, in.partials, in.sc, 3, s);
  CK(cudaMemsetAsync(in.adj_eta, 0, n * 8, s));
  launch_precond(g, in.tabs, in.p.precision, in.r, in.zp, in.work64, in.work32, in.sc, s);
  launch_init_p(g.n, in.zp, in.pv, in.r, in.partials, in.sc, s, g.vec_blocks);
  long long launches = 3 + precond_kernel_count(g);
  DevScalars hs;
  for (;;) {
    CK(cudaMemcpyAsync(&hs, in.sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs.cg_done) break;
    const PcgDot dot{in.r, in.q, in.partials, in.sc, flex};
    const PcgZr zr{in.adj_eta, in.r, in.pv, in.q, in.partials, in.sc};
    launch_ct_hinv(g, in.cf, y, in.pv, nullptr, in.adj_t, s, in.sc);
    launch_apply_C(g, in.adj_t, in.q, 1.0, nullptr, in.partials, in.sc, 2, s, in.pv);
    launch_precond(g, in.tabs, in.p.precision, in.r, in.zp, in.work64, in.work32, in.sc, s, &dot, &zr);
    launch_update_p(g.n, in.zp, in.pv, in.sc, 0, 0, s, g.vec_blocks);
    launches += 3 + precond_step_kernel_count(g, in.tabs);
  }
  // mu = H^{-1}(g - C^T eta), then the contractions
  launch_ct_hinv(g, in.cf, y, in.adj_eta, gy, in.adj_t, s, nullptr);
  launch_adj_grads(g, y, z, in.adj_eta, in.adj_t, dm0, dV, dW, dnu, in.partials, in.sc, s);
  launches += 2;
  pl->launches += launches;
  CK(cudaMemcpyAsync(&hs, in.sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  std::memset(st, 0, sizeof(*st));
  st->status = hs.status;
  st->cg_iters = hs.cg_it;
  st->max_cg_in_solve = hs.cg_it;
  st->r_last = hs.bnorm2 > 0 ? std::sqrt(hs.rr / hs.bnorm2) : 0.0;
  if (hs.status != MFG_OK) return fail(hs.status, "adjoint PCG finished with a non-OK status");
  return MFG_OK;
}

int mfg_apply_precond(mfg_plan_t pl, int b, const double* r, double* z, void* stream) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!r || !z || r == z) return fail(MFG_ERR_INVALID_ARG, "r and z must be distinct non-null arrays");
  Inst& in = pl->inst[b];
  cudaStream_t s = (cudaStream_t)stream;
  launch_precond(in.g, in.tabs, in.p.precision, r, z, in.work64, in.work32, nullptr, s);
  pl->launches += precond_kernel_count(in.g);
  CK(cudaGetLastError());
  return MFG_OK;
}

int mfg_prox(mfg_plan_t pl, int b, double tau, const double* v, const double* V, const double* W,
             double* y, void* stream) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!v || !V || !W || !y) return fail(MFG_ERR_INVALID_ARG, "null array");
  if (!(tau > 0.0)) return fail(MFG_ERR_INVALID_ARG, "tau must be > 0");
  Inst& in = pl->inst[b];
  launch_prox_plain(in.g, in.cf, tau, v, y, V, W, (cudaStream_t)stream);
  pl->launches += 1;
  CK(cudaGetLastError());
  return MFG_OK;
}

int mfg_prox_step(mfg_plan_t pl, int b, double tau, const double* z, double* y, double* ybar,
                  const double* V, const double* W, void* stream) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!z || !y || !ybar || !V || !W) return fail(MFG_ERR_INVALID_ARG, "null array");
  if (y == ybar) return fail(MFG_ERR_INVALID_ARG, "y and ybar must be distinct arrays");
  if (!(tau > 0.0)) return fail(MFG_ERR_INVALID_ARG, "tau must be > 0");
  Inst& in = pl->inst[b];
  DevScalars h{};  // pageable: the copy is staged before cudaMemcpyAsync returns
  h.tau = tau;
  h.sigma = 1.0;
  h.theta = 1.0 / std::sqrt(1.0 + 2.0 * in.p.gamma * tau);
  h.half_itau = 0.5 / tau;
  h.cp_left = 1;
  h.status = MFG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(in.sc, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  launch_prox_cp(in.g, in.cf, z, y, ybar, V, W, in.partials, in.sc, 0, 0, s);
  pl->launches += 1;
  CK(cudaGetLastError());
  return MFG_OK;
}

int mfg_apply_AAt(mfg_plan_t pl, int b, const double* p, double* q, void* stream) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!p || !q || p == q) return fail(MFG_ERR_INVALID_ARG, "p and q must be distinct non-null arrays");
  Inst& in = pl->inst[b];
  launch_AAt(in.g, p, q, in.work64, in.partials, in.sc, 0, (cudaStream_t)stream, in.p.precision == MFG_MIXED_DF);
  pl->launches += aat_kernel_count(in.p.precision == MFG_MIXED_DF);
  CK(cudaGetLastError());
  return MFG_OK;
}

int mfg_apply_C(mfg_plan_t pl, int b, const double* v, double* r, void* stream) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!v || !r) return fail(MFG_ERR_INVALID_ARG, "null array");
  Inst& in = pl->inst[b];
  launch_apply_C(in.g, v, r, 1.0, nullptr, in.partials, in.sc, 0, (cudaStream_t)stream);
  pl->launches += 1;
  CK(cudaGetLastError());
  return MFG_OK;
}

int mfg_apply_Ct(mfg_plan_t pl, int b, const double* p, double* x, void* stream) {
  int rc = check_b(pl, b);
  if (rc != MFG_OK) return rc;
  if (!p || !x) return fail(MFG_ERR_INVALID_ARG, "null array");
  Inst& in = pl->inst[b];
  launch_apply_Ct(in.g, p, x, (cudaStream_t)stream);
  pl->launches += 1;
  CK(cudaGetLastError());
  return MFG_OK;
}

}  // extern "C"
