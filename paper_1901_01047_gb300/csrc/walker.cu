// walker.cu -- host implementation of the C ABI declared in include/dca_walker.h.
//
// The host validates parameters, owns the device memory of all walkers,
// and launches a fixed kernel sequence per submatrix update; all control
// (order, sweep position, measurement and recompute schedule) lives in the
// device-side walker records, so the host reads back only a small status word
// between chunks of windows.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dca_walker.h"
#include "kernels.h"
#include "problem_host.h"
#include "state.h"

using dca::ProblemDev;
using dca::WalkerDev;

namespace {
thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};
}  // namespace

struct dca_walker {
  cudaStream_t stream = nullptr;
  int W = 0, ks = 0, warmup = 0, R = 0, ntm = 0, precision = 0;
  double tie_eps = 1e-10;
  int max_cap = 0, max_nc = 0;
  int q4 = 0;                       // momentum transfer of the two-particle measurement
  std::vector<int> nc_of;           // per walker
  std::vector<size_t> gacc_off;     // per walker offset into the host G layout
  std::vector<WalkerDev> h_W;       // host copies of the walker records
  std::vector<void*> allocs;        // device allocations
  std::vector<uint8_t*> forced;     // per walker replay buffers
  WalkerDev* d_W = nullptr;
  ProblemDev* d_P = nullptr;
  int* d_active = nullptr;          // [8]: active count, -, -, work queues of the inverse (3 .. 6),
                                    // rejected-G0 flag (7)
  int* h_active = nullptr;          // pinned
  int* d_sgn = nullptr;
  dca::Config cfg{};
  dca::TmapDev* d_tmaps = nullptr;  // TMA tensor maps of the tensor-core N update
  std::string err;
  int64_t windows_launched = 0;
  // problem tables (device) for dca_walker_update_G0
  std::vector<ProblemDev> h_P;
  std::vector<double*> g0_stage;    // per problem staging buffer [2][nc][n_tau+1] (slices of one allocation)
  size_t g0_stage_doubles = 0;      // all problems' tables back to back
  long long* d_stage_off = nullptr; // [n_problems] offsets of the slices
  int* d_g0_bad = nullptr;          // [n_problems] per-problem rejection flags of dca_walker_update_G0_all
  int* d_g0_changed = nullptr;      // [n_problems] the last update changed the problem's table
  // timing of kernel groups with CUDA events on the walker's stream
  uint32_t timing_mask = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_pending;  // (group, index of the start event)
  size_t ev_used = 0;
  double group_ms[dca::N_GROUPS] = {0};
  int64_t group_launches[dca::N_GROUPS] = {0};
  int64_t total_launches = 0;
  // device-side window loop: a graph with a conditional WHILE node
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cap_br[4] = {nullptr, nullptr, nullptr, nullptr};  // branches of the captured window
  cudaEvent_t ev_fork = nullptr, ev_join[4] = {nullptr, nullptr, nullptr, nullptr};
  // dca_walker_update_G0_all: the host-to-device copy runs on its own stream,
  // so that it overlaps the sweeps already enqueued; the walker's stream waits
  // for it (staged) and the next copy waits for the commit (stage free)
  cudaStream_t g0_stream = nullptr;
  cudaEvent_t ev_g0_staged = nullptr, ev_g0_free = nullptr;
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  dca::LoopState* d_loop = nullptr;
  dca::LoopState* h_loop = nullptr;  // pinned copy read at synchronisation points
  dca::PoolState* d_pool = nullptr;  // pooled schedule: sweep target and go flag
  int kernels_per_window = 0;
  int64_t loop_iters_seen = 0;       // window-loop iterations already counted
  bool timeout_pending = false;      // a window loop hit its bound since the last dca_walker_sync
  bool g0_rejected = false;          // an update_G0 table had a non-finite entry (reported by sync)
  int64_t max_windows = 0;           // cap of the windows of one sweep call (0 = automatic)
  int prec_public = 0;               // DCA_PREC_* given at create
  double* d_Mout = nullptr;          // read-out of the frequency measurement, all walkers
  long long* d_Mbase = nullptr;      // its per-walker offsets
  double* d_Gout = nullptr;          // read-out of the tau-grid measurement, all walkers back to back
  long long* d_Gbase = nullptr;      // its per-walker offsets (gacc_off)
  double* h_Gout = nullptr;          // pinned host copy of d_Gout (one device-to-host copy per read-out)
  std::vector<int> problem_of;       // per walker

  ~dca_walker() {
    if (stream) cudaStreamSynchronize(stream);
    if (loop_exec) cudaGraphExecDestroy(loop_exec);
    if (loop_graph) cudaGraphDestroy(loop_graph);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (g0_stream) cudaStreamSynchronize(g0_stream);
    if (ev_g0_staged) cudaEventDestroy(ev_g0_staged);
    if (ev_g0_free) cudaEventDestroy(ev_g0_free);
    if (g0_stream) cudaStreamDestroy(g0_stream);
    for (int b = 0; b < 4; ++b) {
      if (ev_join[b]) cudaEventDestroy(ev_join[b]);
      if (cap_br[b]) cudaStreamDestroy(cap_br[b]);
    }
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    for (uint8_t* p : forced)
      if (p) cudaFree(p);
    if (h_active) cudaFreeHost(h_active);
    if (h_loop) cudaFreeHost(h_loop);
    if (h_Gout) cudaFreeHost(h_Gout);
  }

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return p;
  }
};

// The sliced residual lists its tiles (128 x 64 per walker-spin) in the
// 16-bit sub-item field of a persistent CTA's work list; larger capacities
// (n above ~23000) keep the double-float residual.
static bool oz_fits(int cap) { return (long long)((cap + 127) / 128) * ((cap + 63) / 64) < 65536; }

static int fail(dca_walker* w, int code, const std::string& msg) {
  if (w) w->err = msg;
  else g_create_error = msg;
  return code;
}

static int cuda_check(dca_walker* w, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DCA_OK;
  return fail(w, e == cudaErrorMemoryAllocation ? DCA_ERR_OOM : DCA_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                               \
  do {                                                         \
    int _rc = cuda_check(h, (expr), #expr);                    \
    if (_rc != DCA_OK) return _rc;                             \
  } while (0)

extern "C" DCA_API int dca_g0_isolated_cluster(int32_t nc, const double* eps_K, const double* k_dot_r, double mu, double U,
                                       double beta, int32_t n_tau, double* G0_out) {
  if (nc < 1 || n_tau < 1 || !(beta > 0.0) || !eps_K || !k_dot_r || !G0_out)
    return fail(nullptr, DCA_ERR_ARG, "dca_g0_isolated_cluster: invalid argument");
  const size_t m = (size_t)nc * (size_t)(n_tau + 1);
  double *d_eps = nullptr, *d_kr = nullptr, *d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_eps, sizeof(double) * nc);
  if (e == cudaSuccess) e = cudaMalloc(&d_kr, sizeof(double) * nc * nc);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(double) * 2 * m);
  if (e == cudaSuccess) e = cudaMemcpy(d_eps, eps_K, sizeof(double) * nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_kr, k_dot_r, sizeof(double) * nc * nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    dca::launch_g0_isolated(nc, d_eps, d_kr, mu - 0.5 * U, beta, n_tau, d_out, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(G0_out, d_out, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost);
  cudaFree(d_eps);
  cudaFree(d_kr);
  cudaFree(d_out);
  if (e != cudaSuccess) return fail(nullptr, DCA_ERR_CUDA, std::string("dca_g0_isolated_cluster: ") + cudaGetErrorString(e));
  return DCA_OK;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bound of the mbarrier waits of the tensor-core kernels: about two seconds of SM clocks.
constexpr long long kDefaultWaitCycles = 4000000000LL;

static int upload_update_maps(dca_walker* h, int ks, int bn);

extern "C" DCA_API int dca_walker_create(const dca_walker_params* prm, void* cuda_stream, dca_walker** out) {
  if (!out) return fail(nullptr, DCA_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!prm) return fail(nullptr, DCA_ERR_ARG, "params is NULL");
  const dca_walker_params& p = *prm;
  if (p.n_problems < 1 || !p.problems) return fail(nullptr, DCA_ERR_ARG, "need at least one problem");
  if (p.n_walkers < 1) return fail(nullptr, DCA_ERR_ARG, "n_walkers must be >= 1");
  if (p.n_walkers > 16383)  // the work lists of the persistent kernels index walker-spins in 15 bits
    return fail(nullptr, DCA_ERR_ARG, "n_walkers must be <= 16383");
  if (p.k_sub < 1 || p.k_sub > dca::KS_MAX) return fail(nullptr, DCA_ERR_ARG, "k_sub must be in 1..128");
  if (p.recompute_sweeps < 0 || p.recompute_every < 0 || p.warmup_sweeps < 0 || p.n_tau_meas < 1 || p.init_config_size < 0 ||
      p.capacity < 0 || p.log_capacity < 0 || p.recompute_at_measure < 0 || p.recompute_at_measure > 1 ||
      p.n_omega_meas < 0)
    return fail(nullptr, DCA_ERR_ARG, "negative or zero size parameter");
  if (p.precision != DCA_PREC_FP64 && p.precision != DCA_PREC_MIXED && p.precision != DCA_PREC_TF32)
    return fail(nullptr, DCA_ERR_ARG, "unsupported precision");
  if (p.precision == DCA_PREC_TF32 && p.update_kernel == DCA_UPD_CUDA_CORE)
    return fail(nullptr, DCA_ERR_ARG, "DCA_PREC_TF32 runs on the tensor cores only");
  if (!(p.flip_fraction >= 0.0) || p.flip_fraction > 1.0)
    return fail(nullptr, DCA_ERR_ARG, "flip_fraction must be in [0, 1]");
  if (p.duplicate_rule != DCA_DUP_ABORT && p.duplicate_rule != DCA_DUP_NEGLECT && p.duplicate_rule != DCA_DUP_UPDATE)
    return fail(nullptr, DCA_ERR_ARG, "duplicate_rule must be one of DCA_DUP_*");
  if (p.freq_method != DCA_FREQ_NFFT && p.freq_method != DCA_FREQ_DFT)
    return fail(nullptr, DCA_ERR_ARG, "freq_method must be one of DCA_FREQ_*");
  if (p.n_omega_meas != 0 && (p.n_omega_meas < 8 || p.n_omega_meas > 4096))
    return fail(nullptr, DCA_ERR_ARG, "n_omega_meas must be 0 or in 8..4096");
  if (p.gamma_precision != DCA_GAMMA_FP64 && p.gamma_precision != DCA_GAMMA_DOUBLE_FLOAT)
    return fail(nullptr, DCA_ERR_ARG, "gamma_precision must be one of DCA_GAMMA_*");
  if (p.recompute_method < DCA_RECOMPUTE_AUTO || p.recompute_method > DCA_RECOMPUTE_NEWTON_DF)
    return fail(nullptr, DCA_ERR_ARG, "recompute_method must be one of DCA_RECOMPUTE_*");
  if (p.update_kernel < DCA_UPD_AUTO || p.update_kernel > DCA_UPD_TCGEN05)
    return fail(nullptr, DCA_ERR_ARG, "update_kernel must be one of DCA_UPD_*");
  if (p.schedule < DCA_SCHEDULE_LOCKSTEP || p.schedule > DCA_SCHEDULE_POOLED)
    return fail(nullptr, DCA_ERR_ARG, "schedule must be one of DCA_SCHEDULE_*");
  if (p.n_w4 < 0 || p.n_w4 > 32) return fail(nullptr, DCA_ERR_ARG, "n_w4 must be in 0..32");
  if (p.n_w4 > 0 && (p.w4_transfer < -64 || p.w4_transfer > 64))
    return fail(nullptr, DCA_ERR_ARG, "w4_transfer must be in -64..64");
  for (int i = 0; i < p.n_problems; ++i) {
    std::string why;
    if (dca::check_problem(p.problems[i], why) != DCA_OK)
      return fail(nullptr, DCA_ERR_ARG, "problem " + std::to_string(i) + ": " + why);
    if (p.problems[i].nc > 64) return fail(nullptr, DCA_ERR_ARG, "problem " + std::to_string(i) + ": nc > 64");
    if (p.n_w4 > 0) {
      const dca_problem& pr = p.problems[i];
      if (!pr.k_dot_r || !pr.k_sub)
        return fail(nullptr, DCA_ERR_ARG, "problem " + std::to_string(i) + ": the two-particle measurement needs k_dot_r and k_sub");
      if (p.q4_transfer < 0 || p.q4_transfer >= pr.nc)
        return fail(nullptr, DCA_ERR_ARG, "q4_transfer out of range for problem " + std::to_string(i));
      for (int e = 0; e < pr.nc * pr.nc; ++e)
        if (pr.k_sub[e] < 0 || pr.k_sub[e] >= pr.nc || !std::isfinite(pr.k_dot_r[e]))
          return fail(nullptr, DCA_ERR_ARG, "problem " + std::to_string(i) + ": k_sub / k_dot_r out of range");
    }
  }
  if (p.walker_problem)
    for (int w = 0; w < p.n_walkers; ++w)
      if (p.walker_problem[w] < 0 || p.walker_problem[w] >= p.n_problems)
        return fail(nullptr, DCA_ERR_ARG, "walker_problem out of range");

  dca_walker* h = new (std::nothrow) dca_walker();
  if (!h) return fail(nullptr, DCA_ERR_OOM, "host allocation");
  auto bail = [&](int code) {
    g_create_error = h->err;
    delete h;
    return code;
  };
  h->stream = (cudaStream_t)cuda_stream;
  h->W = p.n_walkers;
  h->ks = p.k_sub;
  h->warmup = p.warmup_sweeps;
  h->R = p.recompute_every;
  h->ntm = p.n_tau_meas;
  h->prec_public = p.precision;
  h->precision = p.precision == DCA_PREC_FP64 ? DCA_PREC_FP64 : DCA_PREC_MIXED;  // storage of N
  h->tie_eps = p.tie_eps > 0.0 ? p.tie_eps : 1e-10;

  // ---- problems ----
  std::vector<ProblemDev> hp(p.n_problems);
  for (int i = 0; i < p.n_problems; ++i) {
    const dca_problem& pr = p.problems[i];
    ProblemDev& d = hp[i];
    std::vector<int32_t> add;
    std::vector<double> g0;
    dca::prepare_problem(pr, d, add, g0);
    const size_t tsz = g0.size();
    void* ds = h->dalloc(sizeof(int32_t) * pr.nc * pr.nc);
    void* da = h->dalloc(sizeof(int32_t) * pr.nc * pr.nc);
    void* dg = h->dalloc(sizeof(double) * tsz);
    void* dgf = h->dalloc(sizeof(float) * tsz);
    std::vector<float> g0f(g0.begin(), g0.end());
    if (!ds || !da || !dg || !dgf) {
      h->err = "device allocation of problem tables";
      return bail(DCA_ERR_OOM);
    }
    if (cudaMemcpy(ds, pr.site_sub, sizeof(int32_t) * pr.nc * pr.nc, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(da, add.data(), sizeof(int32_t) * pr.nc * pr.nc, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dg, g0.data(), sizeof(double) * tsz, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dgf, g0f.data(), sizeof(float) * tsz, cudaMemcpyHostToDevice) != cudaSuccess) {
      h->err = "upload of problem tables failed";
      return bail(DCA_ERR_CUDA);
    }
    d.site_sub = (const int32_t*)ds;
    d.site_add = (const int32_t*)da;
    d.g0 = (const double*)dg;
    d.g0f = (const float*)dgf;
    const int q = (p.n_tau_meas > 0 && d.n_tau % p.n_tau_meas == 0) ? d.n_tau / p.n_tau_meas : 0;
    if (h->precision == DCA_PREC_MIXED && q >= 2 && q % 2 == 0) {
      void* dgm = h->dalloc(sizeof(float) * 2 * (size_t)q * pr.nc * (p.n_tau_meas + 1));
      if (!dgm) {
        h->err = "device allocation of the measurement phase table";
        return bail(DCA_ERR_OOM);
      }
      d.g0m = (const float*)dgm;
      d.meas_q = q;
      dca::launch_meas_table(d, p.n_tau_meas, h->stream);
      if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        h->err = "measurement phase table";
        return bail(DCA_ERR_CUDA);
      }
    }
    if (p.n_w4 > 0) {
      // K.r / 2 pi modulo 1 as 56-bit fractions, and the index of Q - K
      std::vector<unsigned long long> kr(pr.nc * pr.nc);
      std::vector<int32_t> kdn(pr.nc);
      for (int e = 0; e < pr.nc * pr.nc; ++e) {
        const double x = pr.k_dot_r[e] / (2.0 * M_PI);
        const double f = x - std::floor(x);
        const double v = std::ldexp(f, 56);
        kr[e] = v >= std::ldexp(1.0, 56) ? 0ull : (unsigned long long)v;
      }
      for (int k = 0; k < pr.nc; ++k) kdn[k] = pr.k_sub[p.q4_transfer * pr.nc + k];
      void* dkr = h->dalloc(sizeof(unsigned long long) * kr.size());
      void* dkd = h->dalloc(sizeof(int32_t) * kdn.size());
      if (!dkr || !dkd) {
        h->err = "device allocation of the two-particle tables";
        return bail(DCA_ERR_OOM);
      }
      if (cudaMemcpy(dkr, kr.data(), sizeof(unsigned long long) * kr.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(dkd, kdn.data(), sizeof(int32_t) * kdn.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        h->err = "upload of the two-particle tables failed";
        return bail(DCA_ERR_CUDA);
      }
      d.kr56 = (const unsigned long long*)dkr;
      d.k_dn = (const int32_t*)dkd;
    }
    h->max_nc = std::max(h->max_nc, pr.nc);
  }
  h->h_P = hp;
  {
    std::vector<long long> soff(p.n_problems);
    for (int i = 0; i < p.n_problems; ++i) {
      soff[i] = (long long)h->g0_stage_doubles;
      h->g0_stage_doubles += (size_t)2 * hp[i].nc * (hp[i].n_tau + 1);
    }
    double* st = (double*)h->dalloc(sizeof(double) * h->g0_stage_doubles);
    h->d_stage_off = (long long*)h->dalloc(sizeof(long long) * p.n_problems);
    h->d_g0_bad = (int*)h->dalloc(sizeof(int) * p.n_problems);
    h->d_g0_changed = (int*)h->dalloc(sizeof(int) * p.n_problems);
    if (!st || !h->d_stage_off || !h->d_g0_bad || !h->d_g0_changed) {
      h->err = "device allocation of G0 staging buffer";
      return bail(DCA_ERR_OOM);
    }
    if (cudaMemcpy(h->d_stage_off, soff.data(), sizeof(long long) * p.n_problems, cudaMemcpyHostToDevice) != cudaSuccess) {
      h->err = "upload of the staging offsets failed";
      return bail(DCA_ERR_CUDA);
    }
    for (int i = 0; i < p.n_problems; ++i) h->g0_stage.push_back(st + soff[i]);
  }
  h->d_P = (ProblemDev*)h->dalloc(sizeof(ProblemDev) * p.n_problems);
  if (!h->d_P || cudaMemcpy(h->d_P, hp.data(), sizeof(ProblemDev) * p.n_problems, cudaMemcpyHostToDevice) != cudaSuccess) {
    h->err = "upload of problem records failed";
    return bail(DCA_ERR_CUDA);
  }

  // ---- walkers ----
  const int KS = dca::KS_MAX;
  // The tensor-core operands exist on every mixed-precision walker, so the
  // update kernel can be switched by dca_walker_set_tuning.
  const bool use_tc = h->precision == DCA_PREC_MIXED && p.update_kernel != DCA_UPD_CUDA_CORE;
  const bool alloc_tc = h->precision == DCA_PREC_MIXED;
  h->h_W.resize(h->W);
  h->nc_of.resize(h->W);
  h->problem_of.resize(h->W);
  h->gacc_off.resize(h->W);
  h->forced.assign(h->W, nullptr);
  size_t goff = 0;
  for (int wi = 0; wi < h->W; ++wi) {
    const int pi = p.walker_problem ? p.walker_problem[wi] : wi % p.n_problems;
    const dca_problem& pr = p.problems[pi];
    int cap = p.capacity;
    if (cap == 0) {
      const double kmax = pr.K + pr.beta * pr.U * pr.nc * 0.5;
      // mean order bound, fluctuations, dead rows awaiting compaction (< 1/8)
      cap = (int)std::ceil(1.5 * kmax) + 2 * p.k_sub + p.init_config_size + 64;
    }
    cap = (int)align_up((size_t)cap, 32);
    if (p.init_config_size + p.k_sub > cap) {
      h->err = "capacity too small for the initial configuration";
      return bail(DCA_ERR_ARG);
    }
    h->max_cap = std::max(h->max_cap, cap);
    h->nc_of[wi] = pr.nc;
    h->problem_of[wi] = pi;
    h->gacc_off[wi] = goff;
    goff += (size_t)2 * pr.nc * p.n_tau_meas;

    WalkerDev& w = h->h_W[wi];
    std::memset(&w, 0, sizeof(w));
    w.cap = cap;
    w.problem = pi;
    w.status = dca::ST_OK;
    w.key0 = (uint32_t)p.seed;
    w.key1 = (uint32_t)(p.seed >> 32) ^ (uint32_t)wi;
    w.sign = 1.0;
    w.log_cap = p.log_capacity;
    const size_t C = (size_t)cap;
    const int nc = pr.nc;
    const size_t esz = h->precision == DCA_PREC_MIXED ? sizeof(float) : sizeof(double);  // N and R
    // one allocation per walker, carved into 256-byte aligned pieces
    struct Piece {
      void** dst;
      size_t bytes;
    };
    std::vector<Piece> pieces;
    for (int par = 0; par < 2; ++par) {
      pieces.push_back({(void**)&w.vsite[par], sizeof(int32_t) * C});
      pieces.push_back({(void**)&w.vtau[par], sizeof(double) * C});
      pieces.push_back({(void**)&w.vs[par], sizeof(int32_t) * C});
      for (int sp = 0; sp < 2; ++sp) pieces.push_back({(void**)&w.N[par][sp], esz * C * C});
    }
    if (h->precision == DCA_PREC_MIXED)
      for (int sp = 0; sp < 2; ++sp) pieces.push_back({(void**)&w.Ascr[sp], sizeof(double) * C * C});
    if (h->precision == DCA_PREC_MIXED && p.recompute_method == DCA_RECOMPUTE_AUTO && oz_fits(cap))
      for (int sp = 0; sp < 2; ++sp) {  // digit planes of the sliced residual (FP16) and their exponents
        pieces.push_back({(void**)&w.OzA[sp], 2 * 5 * C * C});
        pieces.push_back({(void**)&w.OzN[sp], 2 * 4 * C * C});
        pieces.push_back({(void**)&w.OzE[sp], sizeof(int32_t) * 2 * C});
      }
    pieces.push_back({(void**)&w.prop, sizeof(dca::Proposal) * KS});
    for (int sp = 0; sp < 2; ++sp) {
      pieces.push_back({(void**)&w.Gc[sp], sizeof(double) * KS * C});
      pieces.push_back({(void**)&w.Xr[sp], sizeof(double) * KS * C});
      pieces.push_back({(void**)&w.Vb[sp], sizeof(double) * KS * C});
      pieces.push_back({(void**)&w.Ub[sp], sizeof(double) * KS * C});
      pieces.push_back({(void**)&w.Binv[sp], sizeof(double) * KS * KS});
      pieces.push_back({(void**)&w.aP[sp], sizeof(double) * KS});
      pieces.push_back({(void**)&w.Lrow[sp], sizeof(double) * KS * C});
      pieces.push_back({(void**)&w.Lp[sp], sizeof(double) * KS * C});
      pieces.push_back({(void**)&w.Rr[sp], esz * KS * C});
      if (alloc_tc) {
        pieces.push_back({(void**)&w.Aop[sp], sizeof(float) * 2 * C * KS});
        pieces.push_back({(void**)&w.Bop[sp], sizeof(float) * 2 * C * KS});
      }
    }
    pieces.push_back({(void**)&w.P, sizeof(int32_t) * KS});
    pieces.push_back({(void**)&w.removed, sizeof(int32_t) * KS});
    pieces.push_back({(void**)&w.flipped, sizeof(int32_t) * KS});
    pieces.push_back({(void**)&w.acc_slot, sizeof(int32_t) * KS});
    pieces.push_back({(void**)&w.acc_p, sizeof(int32_t) * KS});
    pieces.push_back({(void**)&w.live_idx, sizeof(int32_t) * C});
    pieces.push_back({(void**)&w.surv_tmp, sizeof(int32_t) * C});
    pieces.push_back({(void**)&w.Gacc, sizeof(double) * 2 * nc * p.n_tau_meas});
    pieces.push_back({(void**)&w.Gtmp, sizeof(double) * 2 * nc * p.n_tau_meas});
    pieces.push_back({(void**)&w.gR, sizeof(double) * 2 * nc * C});
    pieces.push_back({(void**)&w.bvec, sizeof(double) * 2 * nc * C});
    if (p.n_omega_meas > 0 || p.n_w4 > 0) pieces.push_back({(void**)&w.vx, sizeof(unsigned long long) * C});
    if (p.n_w4 > 0) {
      const size_t S4 = (size_t)nc * 2 * p.n_w4;
      pieces.push_back({(void**)&w.g4E, 2 * esz * 2 * C * S4});
      pieces.push_back({(void**)&w.g4T, 2 * esz * 2 * C * S4});
      pieces.push_back({(void**)&w.g4A, sizeof(double) * 2 * S4 * S4});
      pieces.push_back({(void**)&w.g4D, sizeof(double) * 4 * S4});
    }
    if (p.n_omega_meas > 0 && p.freq_method == DCA_FREQ_NFFT)
      pieces.push_back({(void**)&w.Mgrid, sizeof(double) * 2 * nc * 4 * (size_t)p.n_omega_meas});
    if (p.n_omega_meas > 0 && p.freq_method == DCA_FREQ_DFT) {
      pieces.push_back({(void**)&w.Mfreq, sizeof(double) * 2 * nc * 2 * (size_t)p.n_omega_meas});
      pieces.push_back({(void**)&w.perm, sizeof(int32_t) * C});
      pieces.push_back({(void**)&w.goff, sizeof(int32_t) * (nc + 1)});
    }
    if (p.log_capacity > 0) pieces.push_back({(void**)&w.log, (size_t)p.log_capacity});
    size_t total = 0;
    for (auto& pc : pieces) total += align_up(pc.bytes, 256);
    char* base = (char*)h->dalloc(total);
    if (!base) {
      h->err = "device allocation of walker " + std::to_string(wi) + " (" + std::to_string(total) + " bytes)";
      return bail(DCA_ERR_OOM);
    }
    if (cudaMemset(base, 0, total) != cudaSuccess) {
      h->err = "cudaMemset failed";
      return bail(DCA_ERR_CUDA);
    }
    size_t off = 0;
    for (auto& pc : pieces) {
      *pc.dst = base + off;
      off += align_up(pc.bytes, 256);
    }
  }
  if (alloc_tc) {
    h->d_tmaps = (dca::TmapDev*)h->dalloc(sizeof(dca::TmapDev) * (size_t)h->W * 2 * dca::TMAPS_PER_SPIN);
    if (!h->d_tmaps || upload_update_maps(h, p.k_sub, h->cfg.upd_bn) != DCA_OK) {
      h->err = "TMA tensor maps of the tensor-core update";
      return bail(DCA_ERR_CUDA);
    }
    if (dca::setup_update_tc() != cudaSuccess || dca::setup_ext_tc() != cudaSuccess ||
        dca::setup_refine_tc() != cudaSuccess) {
      h->err = "tensor-core update kernel attribute setup failed";
      return bail(DCA_ERR_CUDA);
    }
  }
  h->d_W = (WalkerDev*)h->dalloc(sizeof(WalkerDev) * h->W);
  h->d_active = (int*)h->dalloc(sizeof(int) * 8);
  h->d_sgn = (int*)h->dalloc(sizeof(int) * 2 * h->W);
  h->d_pool = (dca::PoolState*)h->dalloc(sizeof(dca::PoolState));
  if (!h->d_W || !h->d_active || !h->d_sgn || !h->d_pool ||
      cudaMallocHost(&h->h_active, sizeof(int) * 4) != cudaSuccess) {
    h->err = "device allocation of walker records";
    return bail(DCA_ERR_OOM);
  }
  if (cudaMemset(h->d_active, 0, sizeof(int) * 8) != cudaSuccess ||
      cudaMemcpy(h->d_W, h->h_W.data(), sizeof(WalkerDev) * h->W, cudaMemcpyHostToDevice) != cudaSuccess) {
    h->err = "upload of walker records";
    return bail(DCA_ERR_CUDA);
  }
  h->cfg.n_walkers = h->W;
  h->cfg.ks = h->ks;
  h->cfg.warmup = h->warmup;
  h->cfg.recompute_every = h->R;
  h->cfg.n_tau_meas = h->ntm;
  h->cfg.prec = h->precision == DCA_PREC_MIXED ? dca::PREC_MIXED : dca::PREC_FP64;
  h->cfg.tie_eps = h->tie_eps;
  h->cfg.W = h->d_W;
  h->cfg.P = h->d_P;
  h->cfg.active_count = h->d_active;
  h->cfg.gj_next = h->d_active + 3;
  h->cfg.recompute_sweeps = p.recompute_sweeps;
  h->cfg.recompute_gj = p.recompute_method == DCA_RECOMPUTE_GJ ? 1 : 0;
  h->cfg.recompute_oz =
      h->precision == DCA_PREC_MIXED && p.recompute_method == DCA_RECOMPUTE_AUTO && oz_fits(h->max_cap) ? 1 : 0;
  h->cfg.upd_kernel = use_tc ? dca::UPD_TCGEN05 : dca::UPD_CUDA_CORE;
  h->cfg.ext_tc = use_tc ? 1 : 0;  // the tcgen05 path covers the G_ext product of the extension too
  h->cfg.tmaps = h->d_tmaps;
  h->cfg.pooled = p.schedule == DCA_SCHEDULE_POOLED ? 1 : 0;
  h->cfg.pool = h->d_pool;
  h->cfg.gamma_fp64 = p.gamma_precision == DCA_GAMMA_FP64 ? 1 : 0;
  h->cfg.tf32_terms = p.precision == DCA_PREC_TF32 ? 1 : 3;
  h->cfg.wait_cycles = kDefaultWaitCycles;
  h->cfg.recompute_at_measure = p.recompute_at_measure ? 1 : 0;
  h->cfg.flip_thr = (uint32_t)std::floor(p.flip_fraction * 1073741824.0);
  h->cfg.dup_rule = p.duplicate_rule;
  h->cfg.n_omega = p.n_omega_meas;
  h->cfg.nfft_L = 4 * p.n_omega_meas;
  h->cfg.nfft_msp = h->precision == DCA_PREC_FP64 ? 12 : 8;
  h->cfg.freq_dft = p.freq_method == DCA_FREQ_DFT ? 1 : 0;
  h->cfg.n_w4 = p.n_w4;
  h->cfg.m4 = p.n_w4 > 0 ? p.w4_transfer : 0;
  h->q4 = p.n_w4 > 0 ? p.q4_transfer : 0;

  if (dca::setup_window_kernels() != cudaSuccess || dca::setup_nfft() != cudaSuccess) {
    h->err = "kernel attribute setup failed";
    return bail(DCA_ERR_CUDA);
  }
  dca::launch_init(h->cfg, p.init_config_size, h->max_cap, h->d_sgn, h->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_W.data(), h->d_W, sizeof(WalkerDev) * h->W, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("initial build: ") + cudaGetErrorString(e);
    return bail(DCA_ERR_CUDA);
  }
  for (int wi = 0; wi < h->W; ++wi)
    if (h->h_W[wi].status != dca::ST_OK) {
      h->err = "initial configuration of walker " + std::to_string(wi) + " is singular";
      return bail(DCA_ERR_NUMERIC);
    }
  *out = h;
  return DCA_OK;
}

// Encode and upload the TMA tensor maps of every walker (the B-operand box
// depends on the submatrix size).
static int upload_update_maps(dca_walker* h, int ks, int bn) {
  std::vector<dca::TmapDev> maps((size_t)h->W * 2 * dca::TMAPS_PER_SPIN);
  for (int wi = 0; wi < h->W; ++wi)
    if (!dca::encode_update_maps(h->h_W[wi], ks, bn, maps.data() + (size_t)wi * 2 * dca::TMAPS_PER_SPIN))
      return DCA_ERR_CUDA;
  if (cudaMemcpy(h->d_tmaps, maps.data(), sizeof(dca::TmapDev) * maps.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return DCA_ERR_CUDA;
  return DCA_OK;
}

static int status_code(int st) {
  switch (st) {
    case dca::ST_OK: return DCA_OK;
    case dca::ST_ERR_NUMERIC: return DCA_ERR_NUMERIC;
    case dca::ST_ERR_CAPACITY: return DCA_ERR_CAPACITY;
    case dca::ST_ERR_TIMEOUT: return DCA_ERR_TIMEOUT;
    default: return DCA_ERR_STATE;
  }
}

// Synchronise the stream and read the walker records, taking stock of the
// device-side window loops run since the last look: their kernel launches,
// and whether a loop hit its iteration bound (kept in h->timeout_pending for
// dca_walker_sync; the device flag is cleared once read).
static int pull_records(dca_walker* h) {
  if (h->d_loop)
    CK(cudaMemcpyAsync(h->h_loop, h->d_loop, sizeof(dca::LoopState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_W.data(), h->d_W, sizeof(WalkerDev) * h->W, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_active + 1, h->d_active + 7, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->h_active[1]) {  // an update_G0 table was rejected on the device
    h->g0_rejected = true;
    CK(cudaMemsetAsync(h->d_active + 7, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  if (h->d_loop) {
    const int64_t it = h->h_loop->total_iters - h->loop_iters_seen;
    h->loop_iters_seen = h->h_loop->total_iters;
    h->windows_launched += it;
    h->total_launches += it * h->kernels_per_window;
    if (h->h_loop->timed_out) {
      h->timeout_pending = true;
      const int32_t zero = 0;
      CK(cudaMemcpyAsync(&h->d_loop->timed_out, &zero, sizeof(zero), cudaMemcpyHostToDevice, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
  }
  return DCA_OK;
}

// First walker error of the pulled records, as a return code with a message.
static int walker_errors(dca_walker* h) {
  for (int wi = 0; wi < h->W; ++wi)
    if (h->h_W[wi].status != dca::ST_OK)
      return fail(h, status_code(h->h_W[wi].status),
                  "walker " + std::to_string(wi) + " stopped with status " + std::to_string(h->h_W[wi].status));
  return DCA_OK;
}

static int push_records(dca_walker* h) {
  CK(cudaMemcpyAsync(h->d_W, h->h_W.data(), sizeof(WalkerDev) * h->W, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return DCA_OK;
}

static cudaEvent_t next_event(dca_walker* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// Whether a window launches the recompute groups (some recompute schedule is set).
static bool has_recompute(const dca_walker* h) {
  return h->R > 0 || h->cfg.recompute_sweeps > 0 || h->cfg.recompute_at_measure;
}

// Launch one kernel group, bracketed by events when its timing bit is set.
// NVTX names of the kernel groups (ranges around each group of the host-driven
// loop, and around the graph launch of the device-side loop), for profilers
// that filter by range.
static const char* const kGroupNames[dca::N_GROUPS] = {
    "dca:propose", "dca:extend",      "dca:metropolis",    "dca:update",       "dca:measure",
    "dca:recompute", "dca:update_pre", "dca:update_post", "dca:recompute_pre", "dca:recompute_post"};

static void run_group(dca_walker* h, int group) {
  nvtxRangePushA(kGroupNames[group]);
  const bool timed = (h->timing_mask >> group) & 1u;
  cudaEvent_t e0 = nullptr;
  size_t i0 = 0;
  if (timed) {
    i0 = h->ev_used;
    e0 = next_event(h);
    if (e0) cudaEventRecord(e0, h->stream);
  }
  int k = 0;
  switch (group) {
    case dca::GROUP_MEASURE: k = dca::launch_measure(h->cfg, h->max_cap, h->max_nc, h->stream); break;
    case dca::GROUP_RECOMPUTE_PRE:
    case dca::GROUP_RECOMPUTE:
    case dca::GROUP_RECOMPUTE_POST: k = dca::launch_recompute(group, h->cfg, h->max_cap, h->d_sgn, h->stream); break;
    default: k = dca::launch_window_group(group, h->cfg, h->max_cap, h->stream); break;
  }
  h->total_launches += k;
  h->group_launches[group] += k;
  if (timed && e0) {
    cudaEvent_t e1 = next_event(h);
    if (e1) {
      cudaEventRecord(e1, h->stream);
      h->ev_pending.push_back({group, (int)i0});
    }
  }
  nvtxRangePop();
}

// After a stream synchronisation: fold the recorded intervals into the totals.
static void collect_events(dca_walker* h) {
  for (auto& pr : h->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[pr.second], h->ev_pool[pr.second + 1]) == cudaSuccess)
      h->group_ms[pr.first] += ms;
  }
  h->ev_pending.clear();
  h->ev_used = 0;
}

// Concurrent branches of the captured window for a batch of W walkers.
static int window_branches(int W) { return W >= 128 ? 4 : (W >= 32 ? 2 : 1); }

// One window's kernel sequence for the walkers of cfg on stream st.
static int launch_window_sequence(dca_walker* h, const dca::Config& cfg, cudaStream_t st) {
  int k = 0;
  for (int i = 0; i < dca::N_WINDOW_GROUPS; ++i) {
    const int g = dca::WINDOW_GROUPS[i];
    if (dca::is_recompute_group(g) && !has_recompute(h)) continue;
    if (g == dca::GROUP_MEASURE)
      k += dca::launch_measure(cfg, h->max_cap, h->max_nc, st);
    else if (g == dca::GROUP_RECOMPUTE_PRE || g == dca::GROUP_RECOMPUTE || g == dca::GROUP_RECOMPUTE_POST)
      k += dca::launch_recompute(g, cfg, h->max_cap, h->d_sgn, st);
    else
      k += dca::launch_window_group(g, cfg, h->max_cap, st);
  }
  return k;
}

// Build the device-side window loop once: an outer graph holding one
// conditional WHILE node whose body (captured from the same launchers the
// host loop uses) is one window plus the loop-control kernel.
static int build_loop_graph(dca_walker* h) {
  if (h->loop_exec) return DCA_OK;
  if (!h->d_loop) {
    h->d_loop = (dca::LoopState*)h->dalloc(sizeof(dca::LoopState));
    if (!h->d_loop) return fail(h, DCA_ERR_OOM, "loop state allocation");
    if (!h->h_loop && cudaMallocHost(&h->h_loop, sizeof(dca::LoopState)) != cudaSuccess)
      return fail(h, DCA_ERR_OOM, "pinned loop state");
    CK(cudaMemsetAsync(h->d_loop, 0, sizeof(dca::LoopState), h->stream));
  }
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CK(cudaGraphCreate(&h->loop_graph, 0));
  cudaGraphConditionalHandle handle;
  CK(cudaGraphConditionalHandleCreate(&handle, h->loop_graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = handle;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, h->loop_graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int k = 0;
  const int nb = window_branches(h->W);
  if (nb > 1) {
    // Independent parts of the batch in concurrent branches of the body: the
    // latency-bound kernels of one part (Metropolis, the factor kernels)
    // overlap the bandwidth- and tensor-bound kernels of the others.
    if (!h->ev_fork) CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventRecord(h->ev_fork, h->cap_stream));
    for (int b = 0; b < nb; ++b) {
      if (!h->cap_br[b]) CK(cudaStreamCreateWithFlags(&h->cap_br[b], cudaStreamNonBlocking));
      if (!h->ev_join[b]) CK(cudaEventCreateWithFlags(&h->ev_join[b], cudaEventDisableTiming));
      const int w0 = (int)((long long)h->W * b / nb), w1 = (int)((long long)h->W * (b + 1) / nb);
      dca::Config cp = h->cfg;
      cp.n_walkers = w1 - w0;
      cp.W = h->cfg.W + w0;
      if (cp.tmaps) cp.tmaps = h->cfg.tmaps + (size_t)w0 * 2 * dca::TMAPS_PER_SPIN;
      cp.gj_next = h->d_active + 3 + b;  // own work queue of the inverse
      CK(cudaStreamWaitEvent(h->cap_br[b], h->ev_fork, 0));
      k += launch_window_sequence(h, cp, h->cap_br[b]);
      CK(cudaEventRecord(h->ev_join[b], h->cap_br[b]));
      CK(cudaStreamWaitEvent(h->cap_stream, h->ev_join[b], 0));
    }
  } else {
    k += launch_window_sequence(h, h->cfg, h->cap_stream);
  }
  dca::launch_loop_control(h->cfg, handle, h->d_loop, h->cap_stream);
  k += 1;
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &captured);
  if (e != cudaSuccess) return cuda_check(h, e, "capture of the window loop");
  CK(cudaGraphInstantiate(&h->loop_exec, h->loop_graph, 0));
  h->kernels_per_window = k;
  return DCA_OK;
}

// Enqueue n_sweeps of the device-side window loop: the sweep target, the
// loop's iteration bound and one graph launch, all stream-ordered.
static int sweep_graph(dca_walker* h, int32_t n_sweeps) {
  int rc = build_loop_graph(h);
  if (rc != DCA_OK) return rc;
  // Every window advances each active walker by >= 1 proposal and a sweep is
  // at most `capacity` proposals, so this bound is never reached normally.
  int64_t max_iters = (int64_t)n_sweeps * (int64_t)(h->max_cap + 1) + 64;
  if (h->max_windows > 0 && h->max_windows < max_iters) max_iters = h->max_windows;
  nvtxRangePushA("dca:sweep_graph");
  dca::launch_add_target(h->cfg, n_sweeps, h->stream);
  dca::launch_loop_reset(h->d_loop, max_iters, h->stream);
  const cudaError_t le = cudaGraphLaunch(h->loop_exec, h->stream);
  nvtxRangePop();
  CK(cudaGetLastError());
  CK(le);
  h->total_launches += 2;
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_sync(dca_walker* h) {
  if (!h) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  if (h->g0_rejected) {
    h->g0_rejected = false;
    return fail(h, DCA_ERR_ARG, "a G0 table given to dca_walker_update_G0 had a non-finite entry; the previous "
                                "table was kept");
  }
  if (h->timeout_pending) {
    h->timeout_pending = false;
    return fail(h, DCA_ERR_TIMEOUT, "window loop reached its iteration bound");
  }
  return walker_errors(h);
}

extern "C" DCA_API int dca_walker_sweep(dca_walker* h, int32_t n_sweeps) {
  if (!h) return DCA_ERR_ARG;
  if (n_sweeps < 0) return fail(h, DCA_ERR_ARG, "n_sweeps < 0");
  if (n_sweeps == 0) return DCA_OK;
  if (h->timing_mask == 0) return sweep_graph(h, n_sweeps);
  // Timed kernel groups: host-driven loop with CUDA events around each group
  // (event nodes are not allowed inside conditional graph bodies).
  dca::launch_add_target(h->cfg, n_sweeps, h->stream);
  h->total_launches += 1;
  CK(cudaGetLastError());
  int chunk = 2;
  for (;;) {
    for (int i = 0; i < chunk; ++i)
      for (int j = 0; j < dca::N_WINDOW_GROUPS; ++j)
        if (!dca::is_recompute_group(dca::WINDOW_GROUPS[j]) || has_recompute(h)) run_group(h, dca::WINDOW_GROUPS[j]);
    h->windows_launched += chunk;
    CK(cudaGetLastError());
    dca::launch_count_active(h->cfg, h->stream);
    h->total_launches += 1;
    CK(cudaMemcpyAsync(h->h_active, h->d_active, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    collect_events(h);
    if (h->h_active[0] == 0) break;
    if (chunk < 64) chunk *= 2;
  }
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  return walker_errors(h);
}

// Drop the captured window loop (it holds the launch configuration by value);
// the next sweep captures it again.
static void drop_loop_graph(dca_walker* h) {
  pull_records(h);  // count the windows of the old graph with its kernels per window
  if (h->loop_exec) {
    cudaGraphExecDestroy(h->loop_exec);
    h->loop_exec = nullptr;
  }
  if (h->loop_graph) {
    cudaGraphDestroy(h->loop_graph);
    h->loop_graph = nullptr;
  }
}

extern "C" DCA_API int dca_walker_set_schedule(dca_walker* h, int32_t schedule) {
  if (!h) return DCA_ERR_ARG;
  if (schedule < DCA_SCHEDULE_LOCKSTEP || schedule > DCA_SCHEDULE_POOLED)
    return fail(h, DCA_ERR_ARG, "schedule must be one of DCA_SCHEDULE_*");
  CK(cudaStreamSynchronize(h->stream));
  h->cfg.pooled = schedule == DCA_SCHEDULE_POOLED ? 1 : 0;
  drop_loop_graph(h);
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_set_recompute(dca_walker* h, int32_t recompute_every, int32_t recompute_sweeps,
                                                int32_t recompute_at_measure) {
  if (!h) return DCA_ERR_ARG;
  if (recompute_every < 0 || recompute_sweeps < 0 || recompute_at_measure < 0 || recompute_at_measure > 1)
    return fail(h, DCA_ERR_ARG, "invalid recompute schedule");
  CK(cudaStreamSynchronize(h->stream));
  h->R = recompute_every;
  h->cfg.recompute_every = recompute_every;
  h->cfg.recompute_sweeps = recompute_sweeps;
  h->cfg.recompute_at_measure = recompute_at_measure;
  drop_loop_graph(h);
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_set_limits(dca_walker* h, int64_t max_windows, int64_t wait_cycles) {
  if (!h) return DCA_ERR_ARG;
  if (max_windows < 0 || wait_cycles < 0) return fail(h, DCA_ERR_ARG, "negative limit");
  CK(cudaStreamSynchronize(h->stream));
  h->max_windows = max_windows;
  h->cfg.wait_cycles = wait_cycles > 0 ? (long long)wait_cycles : kDefaultWaitCycles;
  drop_loop_graph(h);
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_set_tuning(dca_walker* h, int32_t k_sub, int32_t update_kernel) {
  if (!h) return DCA_ERR_ARG;
  if (k_sub < 1 || k_sub > dca::KS_MAX) return fail(h, DCA_ERR_ARG, "k_sub must be in 1..128");
  if (update_kernel < DCA_UPD_AUTO || update_kernel > DCA_UPD_TCGEN05)
    return fail(h, DCA_ERR_ARG, "update_kernel must be one of DCA_UPD_*");
  CK(cudaStreamSynchronize(h->stream));
  const bool mixed = h->cfg.prec == dca::PREC_MIXED;
  const bool tc = mixed && update_kernel != DCA_UPD_CUDA_CORE;
  if (mixed && (dca::tc_tile_n(k_sub, h->cfg.upd_bn) != dca::tc_tile_n(h->ks, h->cfg.upd_bn) ||
                dca::ext_tile_c(k_sub) != dca::ext_tile_c(h->ks))) {
    const int rc = upload_update_maps(h, k_sub, h->cfg.upd_bn);
    if (rc != DCA_OK) return fail(h, rc, "TMA tensor maps of the tensor-core update");
  }
  h->ks = k_sub;
  h->cfg.ks = k_sub;
  h->cfg.upd_kernel = tc ? dca::UPD_TCGEN05 : dca::UPD_CUDA_CORE;
  h->cfg.ext_tc = tc ? 1 : 0;
  drop_loop_graph(h);
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_set_update_tile(dca_walker* h, int32_t tile_n) {
  if (!h) return DCA_ERR_ARG;
  if (tile_n != 0 && tile_n != 32 && tile_n != 64) return fail(h, DCA_ERR_ARG, "tile_n must be 0, 32 or 64");
  if (h->cfg.prec != dca::PREC_MIXED) {
    h->cfg.upd_bn = tile_n;
    return DCA_OK;
  }
  CK(cudaStreamSynchronize(h->stream));
  if (dca::tc_tile_n(h->ks, tile_n) != dca::tc_tile_n(h->ks, h->cfg.upd_bn)) {
    const int rc = upload_update_maps(h, h->ks, tile_n);
    if (rc != DCA_OK) return fail(h, rc, "TMA tensor maps of the tensor-core update");
  }
  h->cfg.upd_bn = tile_n;
  drop_loop_graph(h);
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_set_timing(dca_walker* h, uint32_t group_mask) {
  if (!h) return DCA_ERR_ARG;
  h->timing_mask = group_mask & ((1u << dca::N_GROUPS) - 1u);
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_get_timing(dca_walker* h, double* group_ms, int64_t* group_launches,
                                             int64_t* total_launches, int32_t reset) {
  if (!h) return DCA_ERR_ARG;
  const int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  collect_events(h);
  for (int g = 0; g < dca::N_GROUPS; ++g) {
    if (group_ms) group_ms[g] = h->group_ms[g];
    if (group_launches) group_launches[g] = h->group_launches[g];
  }
  if (total_launches) *total_launches = h->total_launches;
  if (reset) {
    for (int g = 0; g < dca::N_GROUPS; ++g) {
      h->group_ms[g] = 0.0;
      h->group_launches[g] = 0;
    }
    h->total_launches = 0;
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_update_G0(dca_walker* h, int32_t problem, const double* G0) {
  if (!h || problem < 0 || problem >= (int)h->h_P.size() || !G0) return DCA_ERR_ARG;
  const ProblemDev& pd = h->h_P[problem];
  const size_t tsz = (size_t)2 * pd.nc * (pd.n_tau + 1);
  CK(cudaMemcpyAsync(h->g0_stage[problem], G0, sizeof(double) * tsz, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->d_g0_changed, 0, sizeof(int) * h->h_P.size(), h->stream));
  // validated on the device (a table with a non-finite entry is not committed;
  // the next synchronisation reports it)
  dca::launch_negate(h->g0_stage[problem], const_cast<double*>(pd.g0), const_cast<float*>(pd.g0f), tsz,
                     h->d_active + 7, h->d_g0_changed + problem, h->stream);
  h->total_launches += 1;
  if (pd.meas_q > 0) {
    dca::launch_meas_table(pd, h->ntm, h->stream);
    h->total_launches += 1;
  }
  // the staging buffer has been read: a later dca_walker_update_G0_all copy may overwrite it
  if (h->ev_g0_free) CK(cudaEventRecord(h->ev_g0_free, h->stream));
  // N of the walkers on this problem is rebuilt for the new table (only if it changed)
  h->total_launches += dca::launch_rebuild_changed(h->cfg, h->max_cap, h->d_g0_changed, h->d_sgn, h->stream);
  CK(cudaGetLastError());
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_update_G0_all(dca_walker* h, const double* G0_all) {
  if (!h || !G0_all) return DCA_ERR_ARG;
  const int np = (int)h->h_P.size();
  if (!h->g0_stream) {
    CK(cudaStreamCreateWithFlags(&h->g0_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_g0_staged, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_g0_free, cudaEventDisableTiming));
    CK(cudaEventRecord(h->ev_g0_free, h->stream));  // the staging buffers are free after the work enqueued so far
  }
  // the copy overlaps the work already on the walker's stream; the previous
  // commit has read the staging buffers before it starts
  CK(cudaStreamWaitEvent(h->g0_stream, h->ev_g0_free, 0));
  CK(cudaMemcpyAsync(h->g0_stage[0], G0_all, sizeof(double) * h->g0_stage_doubles, cudaMemcpyHostToDevice,
                     h->g0_stream));
  CK(cudaEventRecord(h->ev_g0_staged, h->g0_stream));
  CK(cudaStreamWaitEvent(h->stream, h->ev_g0_staged, 0));
  CK(cudaMemsetAsync(h->d_g0_bad, 0, sizeof(int) * np, h->stream));
  CK(cudaMemsetAsync(h->d_g0_changed, 0, sizeof(int) * np, h->stream));
  dca::launch_g0_update_all(h->d_P, np, h->ntm, h->g0_stage[0], h->d_stage_off, h->d_g0_bad, h->d_active + 7,
                            h->d_g0_changed, h->stream);
  CK(cudaEventRecord(h->ev_g0_free, h->stream));
  h->total_launches += 3;
  h->total_launches += dca::launch_rebuild_changed(h->cfg, h->max_cap, h->d_g0_changed, h->d_sgn, h->stream);
  CK(cudaGetLastError());
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_measure_G(dca_walker* h, double* G_out, double* sign_sum_out, int64_t* n_meas_out) {
  if (!h) return DCA_ERR_ARG;
  if (G_out) {
    // every walker's accumulator gathered on the device into one buffer, one
    // copy to pinned host memory (instead of one small copy per walker)
    const size_t total = (size_t)h->gacc_off[h->W - 1] + (size_t)2 * h->nc_of[h->W - 1] * h->ntm;
    if (!h->d_Gout) {
      h->d_Gout = (double*)h->dalloc(sizeof(double) * total);
      h->d_Gbase = (long long*)h->dalloc(sizeof(long long) * h->W);
      if (!h->d_Gout || !h->d_Gbase) return fail(h, DCA_ERR_OOM, "read-out buffers of the tau-grid measurement");
      if (cudaMallocHost(&h->h_Gout, sizeof(double) * total) != cudaSuccess) {
        h->h_Gout = nullptr;
        cudaGetLastError();
        return fail(h, DCA_ERR_OOM, "pinned read-out buffer of the tau-grid measurement");
      }
      std::vector<long long> base(h->gacc_off.begin(), h->gacc_off.end());
      CK(cudaMemcpyAsync(h->d_Gbase, base.data(), sizeof(long long) * h->W, cudaMemcpyHostToDevice, h->stream));
      CK(cudaStreamSynchronize(h->stream));  // base is a host temporary
    }
    dca::launch_gather_G(h->cfg, h->max_nc, h->d_Gbase, h->d_Gout, h->stream);
    h->total_launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_Gout, h->d_Gout, sizeof(double) * total, cudaMemcpyDeviceToHost, h->stream));
  }
  int rc = pull_records(h);  // synchronises the stream (after the copy above)
  if (rc != DCA_OK) return rc;
  if (G_out) std::memcpy(G_out, h->h_Gout, sizeof(double) * ((size_t)h->gacc_off[h->W - 1] +
                                                            (size_t)2 * h->nc_of[h->W - 1] * h->ntm));
  for (int wi = 0; wi < h->W; ++wi) {
    const WalkerDev& w = h->h_W[wi];
    if (sign_sum_out) sign_sum_out[wi] = w.sign_sum;
    if (n_meas_out) n_meas_out[wi] = w.n_meas;
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_measure_M(dca_walker* h, double* M_out, double* sign_sum_out, int64_t* n_meas_out) {
  if (!h) return DCA_ERR_ARG;
  if (h->cfg.n_omega <= 0) return fail(h, DCA_ERR_STATE, "the frequency measurement is off (n_omega_meas = 0)");
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  const size_t per = (size_t)2 * h->cfg.n_omega * 2;  // spins x frequencies x (re, im), per site difference
  std::vector<long long> base(h->W);
  size_t total = 0;
  for (int wi = 0; wi < h->W; ++wi) {
    base[wi] = (long long)total;
    total += per * h->nc_of[wi];
  }
  if (M_out) {
    if (!h->d_Mout) {
      h->d_Mout = (double*)h->dalloc(sizeof(double) * total);
      h->d_Mbase = (long long*)h->dalloc(sizeof(long long) * h->W);
      if (!h->d_Mout || !h->d_Mbase) return fail(h, DCA_ERR_OOM, "read-out buffers of the frequency measurement");
      CK(cudaMemcpyAsync(h->d_Mbase, base.data(), sizeof(long long) * h->W, cudaMemcpyHostToDevice, h->stream));
    }
    if (h->cfg.freq_dft) dca::launch_ndft_copy(h->cfg, h->max_nc, h->d_Mbase, h->d_Mout, h->stream);
    else dca::launch_nfft_finish(h->cfg, h->max_nc, h->d_Mbase, h->d_Mout, h->stream);
    h->total_launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(M_out, h->d_Mout, sizeof(double) * total, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  for (int wi = 0; wi < h->W; ++wi) {
    if (sign_sum_out) sign_sum_out[wi] = h->h_W[wi].sign_sum;
    if (n_meas_out) n_meas_out[wi] = h->h_W[wi].n_meas;
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_measure_G4(dca_walker* h, double* A_out, double* D_out, double* sign_sum_out,
                                             int64_t* n_meas_out) {
  if (!h) return DCA_ERR_ARG;
  if (h->cfg.n_w4 <= 0) return fail(h, DCA_ERR_STATE, "the two-particle measurement is off (n_w4 = 0)");
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  size_t offA = 0, offD = 0;
  for (int wi = 0; wi < h->W; ++wi) {
    const WalkerDev& w = h->h_W[wi];
    const size_t S4 = (size_t)h->nc_of[wi] * 2 * h->cfg.n_w4;
    if (A_out) CK(cudaMemcpyAsync(A_out + offA, w.g4A, sizeof(double) * 2 * S4 * S4, cudaMemcpyDeviceToHost, h->stream));
    if (D_out) CK(cudaMemcpyAsync(D_out + offD, w.g4D, sizeof(double) * 4 * S4, cudaMemcpyDeviceToHost, h->stream));
    offA += 2 * S4 * S4;
    offD += 4 * S4;
    if (sign_sum_out) sign_sum_out[wi] = w.sign_sum;
    if (n_meas_out) n_meas_out[wi] = w.n_meas;
  }
  CK(cudaStreamSynchronize(h->stream));
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_reset_measurements(dca_walker* h) {
  if (!h) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  for (int wi = 0; wi < h->W; ++wi) {
    WalkerDev& w = h->h_W[wi];
    CK(cudaMemsetAsync(w.Gacc, 0, sizeof(double) * 2 * h->nc_of[wi] * h->ntm, h->stream));
    if (w.Mgrid) CK(cudaMemsetAsync(w.Mgrid, 0, sizeof(double) * 2 * h->nc_of[wi] * h->cfg.nfft_L, h->stream));
    if (w.Mfreq) CK(cudaMemsetAsync(w.Mfreq, 0, sizeof(double) * 4 * h->nc_of[wi] * h->cfg.n_omega, h->stream));
    if (w.g4A) {
      const size_t S4 = (size_t)h->nc_of[wi] * 2 * h->cfg.n_w4;
      CK(cudaMemsetAsync(w.g4A, 0, sizeof(double) * 2 * S4 * S4, h->stream));
      CK(cudaMemsetAsync(w.g4D, 0, sizeof(double) * 4 * S4, h->stream));
    }
    w.sign_sum = 0.0;
    w.n_meas = 0;
    w.k_sum = 0.0;
  }
  return push_records(h);
}

extern "C" DCA_API int dca_walker_stats(dca_walker* h, dca_walker_stats_t* out) {
  if (!h || !out) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  for (int wi = 0; wi < h->W; ++wi) {
    const WalkerDev& w = h->h_W[wi];
    dca_walker_stats_t& s = out[wi];
    s.proposals = w.n_prop;
    s.accepts = w.n_accept;
    s.near_ties = w.n_ties;
    s.aborts = w.n_aborts;
    s.windows = w.n_windows;
    s.sweeps = w.sweeps_done;
    s.measurements = w.n_meas;
    s.recomputes = w.n_recomputes;
    s.sweep_length = w.sweep_len;
    s.order = w.n_live;
    s.status = status_code(w.status);
    s.sign = w.sign;
    s.k_sum = w.k_sum;
    s.max_drift = w.max_drift;
    s.n_update_flops = w.flops;
    s.n_update_bytes = w.upd_bytes;
    s.extend_flops = w.ext_flops;
    s.extend_bytes = w.ext_bytes;
    s.recompute_flops = w.rec_flops;
    s.neglected = w.n_neglected;
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_get_state(dca_walker* h, int32_t wi, dca_vertex* verts, int32_t* k, double* N_up,
                                    double* N_dn) {
  if (!h || wi < 0 || wi >= h->W) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  const WalkerDev& w = h->h_W[wi];
  const int n = w.n, k_live = w.n_live, par = w.parity;
  if (k) *k = k_live;
  if (k_live == 0) return DCA_OK;
  std::vector<int32_t> live(k_live), site(n), s(n);
  std::vector<double> tau(n);
  CK(cudaMemcpyAsync(live.data(), w.live_idx, sizeof(int32_t) * k_live, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(site.data(), w.vsite[par], sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(s.data(), w.vs[par], sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(tau.data(), w.vtau[par], sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (verts)
    for (int i = 0; i < k_live; ++i) {
      verts[i].site = site[live[i]];
      verts[i].s = s[live[i]];
      verts[i].tau = tau[live[i]];
    }
  double* outs[2] = {N_up, N_dn};
  const bool f32 = h->cfg.prec == dca::PREC_MIXED;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  std::vector<unsigned char> full((size_t)n * n * esz);
  for (int sp = 0; sp < 2; ++sp) {
    if (!outs[sp]) continue;
    CK(cudaMemcpy2DAsync(full.data(), esz * n, w.N[par][sp], esz * w.cap, esz * n, n, cudaMemcpyDeviceToHost,
                         h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < k_live; ++i)
      for (int j = 0; j < k_live; ++j) {
        const size_t o = (size_t)live[i] * n + live[j];
        outs[sp][(size_t)i * k_live + j] = f32 ? (double)((const float*)full.data())[o] : ((const double*)full.data())[o];
      }
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_get_decision_log(dca_walker* h, int32_t wi, uint8_t* out, int64_t cap, int64_t* n) {
  if (!h || wi < 0 || wi >= h->W) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  const WalkerDev& w = h->h_W[wi];
  const int64_t logged = (int64_t)w.q < w.log_cap ? (int64_t)w.q : w.log_cap;
  if (n) *n = (int64_t)w.q;
  if (out && cap > 0 && logged > 0) {
    CK(cudaMemcpyAsync(out, w.log, (size_t)(logged < cap ? logged : cap), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_set_forced_decisions(dca_walker* h, int32_t wi, const uint8_t* log, int64_t n) {
  if (!h || wi < 0 || wi >= h->W || n < 0 || (n > 0 && !log)) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  if (h->forced[wi]) {
    cudaFree(h->forced[wi]);
    h->forced[wi] = nullptr;
  }
  WalkerDev& w = h->h_W[wi];
  w.forced = nullptr;
  w.forced_n = 0;
  if (n > 0) {
    uint8_t* d = nullptr;
    CK(cudaMalloc(&d, (size_t)n));
    h->forced[wi] = d;
    CK(cudaMemcpy(d, log, (size_t)n, cudaMemcpyHostToDevice));
    w.forced = d;
    w.forced_n = n;
  }
  return push_records(h);
}

// ---------------------------------------------------------------------------
// Checkpoint / resume.  Layout: SaveHeader, then per walker a SaveWalker
// record, its k vertices (SaveVertex), its G accumulator [2][nc][n_tau_meas]
// and, with the frequency measurement on, its NFFT grid [2][nc][4 n_omega]
// or dense sums [2][nc][n_omega][2], with the two-particle measurement on, its
// accumulators [S][S][2] and [2][S][2] (FP64), all little-endian host structs of
// fixed layout.
// ---------------------------------------------------------------------------
namespace {
constexpr uint32_t kSaveMagic = 0x57414344u;  // "DCAW"
constexpr uint32_t kSaveVersion = 4u;

struct SaveHeader {
  uint32_t magic, version;
  int32_t n_walkers, precision, n_tau_meas, warmup, n_omega, freq_dft, n_w4, w4_transfer, q4_transfer, pad;
  uint64_t bytes;  // total size of the checkpoint
};

struct SaveWalker {
  int32_t problem, nc, k, status;
  int32_t windows_since_recompute, pad;
  uint64_t q;
  int64_t sweeps_done, sweep_pos, sweep_len_cur, sweep_len, warm_k_sum;
  int64_t n_prop, n_accept, n_ties, n_aborts, n_windows, n_meas, n_recomputes, n_neglected;
  double sign, sign_sum, k_sum, max_drift, flops, upd_bytes, ext_flops, ext_bytes, rec_flops;
};

struct SaveVertex {
  int32_t site, s;
  double tau;
};
}  // namespace

// Bytes of a walker's accumulators in a checkpoint: G(tau), then the
// frequency measurement's (the NFFT grid or the dense sums).
static size_t freq_acc_doubles(const dca_walker* h, int wi) {
  if (h->cfg.n_omega <= 0) return 0;
  return (size_t)h->nc_of[wi] * (h->cfg.freq_dft ? 4 * (size_t)h->cfg.n_omega : 2 * (size_t)h->cfg.nfft_L);
}

static size_t g4_acc_doubles(const dca_walker* h, int wi) {
  if (h->cfg.n_w4 <= 0) return 0;
  const size_t S4 = (size_t)h->nc_of[wi] * 2 * h->cfg.n_w4;
  return 2 * S4 * S4 + 4 * S4;
}

static size_t acc_bytes(const dca_walker* h, int wi) {
  return sizeof(double) * (2 * (size_t)h->nc_of[wi] * (size_t)h->ntm + freq_acc_doubles(h, wi) + g4_acc_doubles(h, wi));
}

// The device accumulators of a walker in checkpoint order (pointer, bytes).
static std::vector<std::pair<double*, size_t>> acc_segments(const dca_walker* h, int wi) {
  const WalkerDev& w = h->h_W[wi];
  std::vector<std::pair<double*, size_t>> seg;
  seg.push_back({w.Gacc, sizeof(double) * 2 * (size_t)h->nc_of[wi] * h->ntm});
  if (w.Mgrid || w.Mfreq) seg.push_back({w.Mgrid ? w.Mgrid : w.Mfreq, sizeof(double) * freq_acc_doubles(h, wi)});
  if (w.g4A) {
    const size_t S4 = (size_t)h->nc_of[wi] * 2 * h->cfg.n_w4;
    seg.push_back({w.g4A, sizeof(double) * 2 * S4 * S4});
    seg.push_back({w.g4D, sizeof(double) * 4 * S4});
  }
  return seg;
}

static size_t save_size(const dca_walker* h) {
  size_t b = sizeof(SaveHeader);
  for (int wi = 0; wi < h->W; ++wi)
    b += sizeof(SaveWalker) + sizeof(SaveVertex) * (size_t)h->h_W[wi].n_live + acc_bytes(h, wi);
  return b;
}

extern "C" DCA_API int dca_walker_save(dca_walker* h, void* buf, size_t cap, size_t* n) {
  if (!h || !n) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  const size_t need = save_size(h);
  *n = need;
  if (!buf) return DCA_OK;
  if (cap < need) return fail(h, DCA_ERR_ARG, "checkpoint buffer too small (" + std::to_string(need) + " bytes needed)");
  unsigned char* out = (unsigned char*)buf;
  SaveHeader hd{kSaveMagic,       kSaveVersion, h->W,      h->prec_public, h->ntm, h->warmup, h->cfg.n_omega,
                h->cfg.freq_dft, h->cfg.n_w4,  h->cfg.m4, h->q4,          0,      (uint64_t)need};
  std::memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  for (int wi = 0; wi < h->W; ++wi) {
    const WalkerDev& w = h->h_W[wi];
    const int k = w.n_live, n_rows = w.n, par = w.parity;
    SaveWalker sw{};
    sw.problem = h->problem_of[wi];
    sw.nc = h->nc_of[wi];
    sw.k = k;
    sw.status = w.status;
    sw.windows_since_recompute = w.windows_since_recompute;
    sw.q = w.q;
    sw.sweeps_done = w.sweeps_done;
    sw.sweep_pos = w.sweep_pos;
    sw.sweep_len_cur = w.sweep_len_cur;
    sw.sweep_len = w.sweep_len;
    sw.warm_k_sum = w.warm_k_sum;
    sw.n_prop = w.n_prop;
    sw.n_accept = w.n_accept;
    sw.n_ties = w.n_ties;
    sw.n_aborts = w.n_aborts;
    sw.n_windows = w.n_windows;
    sw.n_meas = w.n_meas;
    sw.n_recomputes = w.n_recomputes;
    sw.n_neglected = w.n_neglected;
    sw.sign = w.sign;
    sw.sign_sum = w.sign_sum;
    sw.k_sum = w.k_sum;
    sw.max_drift = w.max_drift;
    sw.flops = w.flops;
    sw.upd_bytes = w.upd_bytes;
    sw.ext_flops = w.ext_flops;
    sw.ext_bytes = w.ext_bytes;
    sw.rec_flops = w.rec_flops;
    std::memcpy(out + off, &sw, sizeof(sw));
    off += sizeof(sw);
    std::vector<int32_t> live(k), site(n_rows), s(n_rows);
    std::vector<double> tau(n_rows);
    if (k > 0) {
      CK(cudaMemcpyAsync(live.data(), w.live_idx, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(site.data(), w.vsite[par], sizeof(int32_t) * n_rows, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(s.data(), w.vs[par], sizeof(int32_t) * n_rows, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(tau.data(), w.vtau[par], sizeof(double) * n_rows, cudaMemcpyDeviceToHost, h->stream));
    }
    size_t aoff = off + sizeof(SaveVertex) * k;
    for (const auto& sg : acc_segments(h, wi)) {
      CK(cudaMemcpyAsync(out + aoff, sg.first, sg.second, cudaMemcpyDeviceToHost, h->stream));
      aoff += sg.second;
    }
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < k; ++i) {
      const SaveVertex v{site[live[i]], s[live[i]], tau[live[i]]};
      std::memcpy(out + off + sizeof(SaveVertex) * i, &v, sizeof(v));
    }
    off += sizeof(SaveVertex) * k + acc_bytes(h, wi);
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_load(dca_walker* h, const void* buf, size_t n) {
  if (!h || !buf) return DCA_ERR_ARG;
  int rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  const unsigned char* in = (const unsigned char*)buf;
  SaveHeader hd;
  if (n < sizeof(hd)) return fail(h, DCA_ERR_ARG, "checkpoint truncated");
  std::memcpy(&hd, in, sizeof(hd));
  if (hd.magic != kSaveMagic || hd.version != kSaveVersion) return fail(h, DCA_ERR_ARG, "not a walker checkpoint");
  if (hd.bytes != n) return fail(h, DCA_ERR_ARG, "checkpoint size does not match its header");
  if (hd.n_walkers != h->W || hd.precision != h->prec_public || hd.n_tau_meas != h->ntm || hd.warmup != h->warmup ||
      hd.n_omega != h->cfg.n_omega || hd.freq_dft != h->cfg.freq_dft || hd.n_w4 != h->cfg.n_w4 ||
      hd.w4_transfer != h->cfg.m4 || hd.q4_transfer != h->q4)
    return fail(h, DCA_ERR_ARG, "checkpoint of a walker set with other parameters");
  // first pass: validate everything before touching the walkers
  struct Parsed {
    SaveWalker sw;
    size_t vert_off, g_off;
  };
  std::vector<Parsed> parsed(h->W);
  size_t off = sizeof(hd);
  int max_k = 0;
  for (int wi = 0; wi < h->W; ++wi) {
    if (off + sizeof(SaveWalker) > n) return fail(h, DCA_ERR_ARG, "checkpoint truncated");
    Parsed& p = parsed[wi];
    std::memcpy(&p.sw, in + off, sizeof(SaveWalker));
    off += sizeof(SaveWalker);
    const SaveWalker& sw = p.sw;
    const WalkerDev& w = h->h_W[wi];
    if (sw.problem != h->problem_of[wi] || sw.nc != h->nc_of[wi])
      return fail(h, DCA_ERR_ARG, "walker " + std::to_string(wi) + ": checkpoint of another problem");
    if (sw.k < 0 || sw.k + h->ks > w.cap)
      return fail(h, DCA_ERR_ARG, "walker " + std::to_string(wi) + ": order beyond the capacity");
    if (sw.sign != 1.0 && sw.sign != -1.0) return fail(h, DCA_ERR_ARG, "walker " + std::to_string(wi) + ": bad sign");
    p.vert_off = off;
    p.g_off = off + sizeof(SaveVertex) * (size_t)sw.k;
    off = p.g_off + acc_bytes(h, wi);
    if (off > n) return fail(h, DCA_ERR_ARG, "checkpoint truncated");
    const ProblemDev& pd = h->h_P[sw.problem];
    for (int i = 0; i < sw.k; ++i) {
      SaveVertex v;
      std::memcpy(&v, in + p.vert_off + sizeof(SaveVertex) * i, sizeof(v));
      if (v.site < 0 || v.site >= pd.nc || (v.s != 1 && v.s != -1) || !(v.tau >= 0.0) || !(v.tau < pd.beta))
        return fail(h, DCA_ERR_ARG, "walker " + std::to_string(wi) + ": vertex " + std::to_string(i) + " out of range");
    }
    max_k = std::max(max_k, sw.k);
  }
  if (off != n) return fail(h, DCA_ERR_ARG, "checkpoint has trailing bytes");
  // second pass: upload the configurations and counters
  for (int wi = 0; wi < h->W; ++wi) {
    const Parsed& p = parsed[wi];
    const SaveWalker& sw = p.sw;
    WalkerDev& w = h->h_W[wi];
    const int k = sw.k;
    std::vector<int32_t> site(k), s(k), live(k);
    std::vector<double> tau(k);
    for (int i = 0; i < k; ++i) {
      SaveVertex v;
      std::memcpy(&v, in + p.vert_off + sizeof(SaveVertex) * i, sizeof(v));
      site[i] = v.site;
      s[i] = v.s;
      tau[i] = v.tau;
      live[i] = i;
    }
    if (k > 0) {
      CK(cudaMemcpyAsync(w.vsite[0], site.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(w.vs[0], s.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(w.vtau[0], tau.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(w.live_idx, live.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, h->stream));
    }
    size_t aoff = p.g_off;
    for (const auto& sg : acc_segments(h, wi)) {
      CK(cudaMemcpyAsync(sg.first, in + aoff, sg.second, cudaMemcpyHostToDevice, h->stream));
      aoff += sg.second;
    }
    CK(cudaMemsetAsync(w.Gtmp, 0, sizeof(double) * 2 * (size_t)sw.nc * h->ntm, h->stream));
    w.n = k;
    w.n_live = k;
    w.n_dead = 0;
    w.compact_pending = 0;
    w.parity = 0;
    w.status = sw.status;
    w.windows_since_recompute = sw.windows_since_recompute;
    w.q = sw.q;
    w.sweeps_done = sw.sweeps_done;
    w.sweeps_target = sw.sweeps_done;
    w.sweeps_base = sw.sweeps_done;
    w.sweep_pos = sw.sweep_pos;
    w.sweep_len_cur = sw.sweep_len_cur;
    w.sweep_len = sw.sweep_len;
    w.warm_k_sum = sw.warm_k_sum;
    w.n_prop = sw.n_prop;
    w.n_accept = sw.n_accept;
    w.n_ties = sw.n_ties;
    w.n_aborts = sw.n_aborts;
    w.n_windows = sw.n_windows;
    w.n_meas = sw.n_meas;
    w.n_recomputes = sw.n_recomputes;
    w.n_neglected = sw.n_neglected;
    w.sign = sw.sign;
    w.sign_sum = sw.sign_sum;
    w.k_sum = sw.k_sum;
    w.max_drift = sw.max_drift;
    w.drift_bits[0] = w.drift_bits[1] = 0ull;
    w.flops = sw.flops;
    w.upd_bytes = sw.upd_bytes;
    w.ext_flops = sw.ext_flops;
    w.ext_bytes = sw.ext_bytes;
    w.rec_flops = sw.rec_flops;
    w.active = 0;
    w.win_len = w.n_cand = w.n_acc = w.n_removed = w.n_eval = w.aborted = w.n_ins = 0;
    w.measure_pending = w.recompute_pending = w.first_window = 0;
  }
  rc = push_records(h);
  if (rc != DCA_OK) return rc;
  dca::launch_rebuild(h->cfg, max_k, h->d_sgn, h->stream);
  CK(cudaGetLastError());
  rc = pull_records(h);
  if (rc != DCA_OK) return rc;
  for (int wi = 0; wi < h->W; ++wi) {
    WalkerDev& w = h->h_W[wi];
    if (w.n_live > 0 && w.sign != parsed[wi].sw.sign)
      return fail(h, DCA_ERR_NUMERIC, "walker " + std::to_string(wi) + ": rebuilt determinant sign differs from the saved sign");
    if (w.status == dca::ST_ERR_NUMERIC && parsed[wi].sw.status == dca::ST_OK)
      return fail(h, DCA_ERR_NUMERIC, "walker " + std::to_string(wi) + ": rebuilt matrix is singular");
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_walker_capacity(dca_walker* h, int32_t wi, int32_t* capacity) {
  if (!h || wi < 0 || wi >= h->W || !capacity) return DCA_ERR_ARG;
  *capacity = h->h_W[wi].cap;
  return DCA_OK;
}

extern "C" DCA_API void dca_walker_destroy(dca_walker* h) { delete h; }

extern "C" DCA_API const char* dca_walker_last_error(dca_walker* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

// ---------------------------------------------------------------------------
// Standalone from-scratch N (the periodic recompute as its own operation).
// ---------------------------------------------------------------------------
int dca_check_vertices(const dca_problem& pr, int32_t n, const dca_vertex* verts, std::string& err) {
  if (n < 0 || (n > 0 && !verts)) {
    err = "invalid vertex list";
    return DCA_ERR_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const dca_vertex& v = verts[i];
    if (v.site < 0 || v.site >= pr.nc || (v.s != 1 && v.s != -1) || !(v.tau >= 0.0) || !(v.tau < pr.beta)) {
      err = "vertex " + std::to_string(i) + " out of range";
      return DCA_ERR_ARG;
    }
  }
  return DCA_OK;
}

extern "C" DCA_API int dca_fresh_N(const dca_problem* problem, int32_t n, const dca_vertex* verts, double* N_up,
                                   double* N_dn, int32_t* det_sign) {
  if (!problem) return fail(nullptr, DCA_ERR_ARG, "dca_fresh_N: problem is NULL");
  std::string why;
  if (dca::check_problem(*problem, why) != DCA_OK || dca_check_vertices(*problem, n, verts, why) != DCA_OK)
    return fail(nullptr, DCA_ERR_ARG, "dca_fresh_N: " + why);
  if (n == 0) {
    if (det_sign) *det_sign = 1;
    return DCA_OK;
  }
  const dca_problem& pr = *problem;
  ProblemDev d{};
  std::vector<int32_t> add;
  std::vector<double> g0;
  dca::prepare_problem(pr, d, add, g0);
  const size_t nn = (size_t)n * n, nc2 = (size_t)pr.nc * pr.nc;
  struct Piece {
    void** dst;
    size_t bytes;
  };
  int32_t *d_ss, *d_sa, *d_site, *d_s, *d_sgn;
  double *d_g0, *d_tau, *d_N[2], *d_scr[2];
  ProblemDev* d_P;
  WalkerDev* d_W;
  std::vector<Piece> pieces = {{(void**)&d_ss, sizeof(int32_t) * nc2},   {(void**)&d_sa, sizeof(int32_t) * nc2},
                               {(void**)&d_g0, sizeof(double) * g0.size()}, {(void**)&d_P, sizeof(ProblemDev)},
                               {(void**)&d_W, sizeof(WalkerDev)},          {(void**)&d_site, sizeof(int32_t) * n},
                               {(void**)&d_tau, sizeof(double) * n},       {(void**)&d_s, sizeof(int32_t) * n},
                               {(void**)&d_N[0], sizeof(double) * nn},     {(void**)&d_N[1], sizeof(double) * nn},
                               {(void**)&d_scr[0], sizeof(double) * 2 * n}, {(void**)&d_scr[1], sizeof(double) * 2 * n},
                               {(void**)&d_sgn, sizeof(int32_t) * 4}};
  size_t total = 0;
  for (auto& pc : pieces) total += align_up(pc.bytes, 256);
  char* base = nullptr;
  cudaError_t e = cudaMalloc(&base, total);
  if (e != cudaSuccess) return fail(nullptr, DCA_ERR_OOM, std::string("dca_fresh_N: ") + cudaGetErrorString(e));
  size_t off = 0;
  for (auto& pc : pieces) {
    *pc.dst = base + off;
    off += align_up(pc.bytes, 256);
  }
  d.site_sub = d_ss;
  d.site_add = d_sa;
  d.g0 = d_g0;
  WalkerDev w;
  std::memset(&w, 0, sizeof(w));
  w.n = n;
  w.cap = n;
  w.status = dca::ST_OK;
  w.sign = 1.0;
  w.vsite[0] = d_site;
  w.vtau[0] = d_tau;
  w.vs[0] = d_s;
  w.N[0][0] = d_N[0];
  w.N[0][1] = d_N[1];
  w.Lrow[0] = d_scr[0];
  w.Lrow[1] = d_scr[1];
  std::vector<int32_t> site(n), s(n);
  std::vector<double> tau(n);
  for (int i = 0; i < n; ++i) {
    site[i] = verts[i].site;
    s[i] = verts[i].s;
    tau[i] = verts[i].tau;
  }
  dca::Config cfg{};
  cfg.n_walkers = 1;
  cfg.W = d_W;
  cfg.P = d_P;
  cfg.gj_next = d_sgn + 2;  // work queue of the inverse
  int32_t sgn[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(d_ss, pr.site_sub, sizeof(int32_t) * nc2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_sa, add.data(), sizeof(int32_t) * nc2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_g0, g0.data(), sizeof(double) * g0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_P, &d, sizeof(ProblemDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_W, &w, sizeof(WalkerDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_site, site.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_tau, tau.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_s, s.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    dca::launch_fresh_inverse(cfg, n, d_sgn, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(sgn, d_sgn, sizeof(sgn), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && N_up) e = cudaMemcpy(N_up, d_N[0], sizeof(double) * nn, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && N_dn) e = cudaMemcpy(N_dn, d_N[1], sizeof(double) * nn, cudaMemcpyDeviceToHost);
  cudaFree(base);
  if (e != cudaSuccess) return fail(nullptr, DCA_ERR_CUDA, std::string("dca_fresh_N: ") + cudaGetErrorString(e));
  if (sgn[0] == 0 || sgn[1] == 0) return fail(nullptr, DCA_ERR_NUMERIC, "dca_fresh_N: singular matrix");
  if (det_sign) *det_sign = sgn[0] * sgn[1];
  return DCA_OK;
}

namespace dca {
void set_handleless_error(const std::string& msg) { g_create_error = msg; }
}  // namespace dca
