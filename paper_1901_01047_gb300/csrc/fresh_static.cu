// fresh_static.cu -- from-scratch N with no device allocation at all.
//
// dca_fresh_N allocates its device buffers for each call.  Some callers cannot
// let a library allocate device memory: processes whose device memory is
// owned by another allocator (for example a framework's caching allocator
// that has reserved the pool), and services that must keep their device
// footprint fixed after start-up.  For them,
// dca_fresh_N_noalloc does the same work with every device buffer carved out
// of one file-scope __device__ array of fixed size (about 3.2 MB, held by
// every GPU that loads the library until the process exits).
//
// Host code only ever sees a host-side stand-in for the array's name; the
// device address comes from cudaGetSymbolAddress, looked up once per device
// (with that device current) on the first call made on it.  Make that first
// call before any stream capture begins.  The address is kept for the life of
// the process; a cudaDeviceReset frees the array's storage, so the function
// must not be called again after a reset.
//
// The array is shared by every call and keeps the last call's contents.  This
// entry point serialises its own callers with a mutex and uses synchronous
// copies on the legacy default stream, but work that overlaps it on the GPU
// from elsewhere in the process (kernels reading the array, another copy of
// this library's state) races with it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dca_walker.h"
#include "kernels.h"
#include "problem_host.h"
#include "state.h"

namespace {

constexpr int kMaxOrder = DCA_NOALLOC_MAX_ORDER;            // n
constexpr int kMaxSites = DCA_NOALLOC_MAX_SITES;            // nc
constexpr size_t kMaxTable = DCA_NOALLOC_MAX_TABLE;         // 2 * nc * (n_tau + 1) doubles

constexpr size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Fixed layout of the scratch array (every piece 256-byte aligned).
constexpr size_t kOffSiteSub = 0;
constexpr size_t kOffSiteAdd = kOffSiteSub + up256(sizeof(int32_t) * kMaxSites * kMaxSites);
constexpr size_t kOffG0 = kOffSiteAdd + up256(sizeof(int32_t) * kMaxSites * kMaxSites);
constexpr size_t kOffProblem = kOffG0 + up256(sizeof(double) * kMaxTable);
constexpr size_t kOffWalker = kOffProblem + up256(sizeof(dca::ProblemDev));
constexpr size_t kOffSite = kOffWalker + up256(sizeof(dca::WalkerDev));
constexpr size_t kOffTau = kOffSite + up256(sizeof(int32_t) * kMaxOrder);
constexpr size_t kOffSpin = kOffTau + up256(sizeof(double) * kMaxOrder);
constexpr size_t kOffN0 = kOffSpin + up256(sizeof(int32_t) * kMaxOrder);
constexpr size_t kOffN1 = kOffN0 + up256(sizeof(double) * kMaxOrder * kMaxOrder);
constexpr size_t kOffScr0 = kOffN1 + up256(sizeof(double) * kMaxOrder * kMaxOrder);
constexpr size_t kOffScr1 = kOffScr0 + up256(sizeof(double) * 2 * kMaxOrder);
constexpr size_t kOffSign = kOffScr1 + up256(sizeof(double) * 2 * kMaxOrder);
constexpr size_t kScratchBytes = kOffSign + up256(sizeof(int32_t) * 4);  // two signs, work queue

static __device__ __align__(256) unsigned char g_fresh_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
unsigned char* g_addr[kMaxDevices] = {nullptr};

int fail(int code, const std::string& msg) {
  dca::set_handleless_error("dca_fresh_N_noalloc: " + msg);
  return code;
}

}  // namespace

extern "C" DCA_API int dca_fresh_N_noalloc(const dca_problem* problem, int32_t n, const dca_vertex* verts,
                                           double* N_up, double* N_dn, int32_t* det_sign) {
  if (!problem) return fail(DCA_ERR_ARG, "problem is NULL");
  std::string why;
  if (dca::check_problem(*problem, why) != DCA_OK) return fail(DCA_ERR_ARG, why);
  const dca_problem& pr = *problem;
  if (n < 0 || (n > 0 && !verts)) return fail(DCA_ERR_ARG, "invalid vertex list");
  for (int i = 0; i < n; ++i) {
    const dca_vertex& v = verts[i];
    if (v.site < 0 || v.site >= pr.nc || (v.s != 1 && v.s != -1) || !(v.tau >= 0.0) || !(v.tau < pr.beta))
      return fail(DCA_ERR_ARG, "vertex " + std::to_string(i) + " out of range");
  }
  const size_t table = (size_t)2 * pr.nc * (size_t)(pr.n_tau + 1);
  if (n > kMaxOrder || pr.nc > kMaxSites || table > kMaxTable)
    return fail(DCA_ERR_ARG, "size beyond the fixed scratch: order " + std::to_string(n) + " (max " +
                                 std::to_string(kMaxOrder) + "), sites " + std::to_string(pr.nc) + " (max " +
                                 std::to_string(kMaxSites) + "), G0 table " + std::to_string(table) +
                                 " doubles (max " + std::to_string(kMaxTable) + ")");
  if (n == 0) {
    if (det_sign) *det_sign = 1;
    return DCA_OK;
  }

  std::lock_guard<std::mutex> guard(g_lock);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DCA_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(DCA_ERR_ARG, "device index beyond " + std::to_string(kMaxDevices));
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fresh_scratch);
    if (e != cudaSuccess || !p) return fail(DCA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = (unsigned char*)p;
  }
  unsigned char* base = g_addr[dev];

  dca::ProblemDev d{};
  std::vector<int32_t> add;
  std::vector<double> g0;
  dca::prepare_problem(pr, d, add, g0);
  d.site_sub = (const int32_t*)(base + kOffSiteSub);
  d.site_add = (const int32_t*)(base + kOffSiteAdd);
  d.g0 = (const double*)(base + kOffG0);

  dca::WalkerDev w;
  std::memset(&w, 0, sizeof(w));
  w.n = n;
  w.cap = n;
  w.status = dca::ST_OK;
  w.sign = 1.0;
  w.vsite[0] = (int32_t*)(base + kOffSite);
  w.vtau[0] = (double*)(base + kOffTau);
  w.vs[0] = (int32_t*)(base + kOffSpin);
  w.N[0][0] = (double*)(base + kOffN0);
  w.N[0][1] = (double*)(base + kOffN1);
  w.Lrow[0] = (double*)(base + kOffScr0);
  w.Lrow[1] = (double*)(base + kOffScr1);
  int32_t* d_sgn = (int32_t*)(base + kOffSign);

  std::vector<int32_t> site(n), s(n);
  std::vector<double> tau(n);
  for (int i = 0; i < n; ++i) {
    site[i] = verts[i].site;
    s[i] = verts[i].s;
    tau[i] = verts[i].tau;
  }
  dca::Config cfg{};
  cfg.n_walkers = 1;
  cfg.W = (dca::WalkerDev*)(base + kOffWalker);
  cfg.P = (const dca::ProblemDev*)(base + kOffProblem);
  cfg.gj_next = d_sgn + 2;  // work queue of the inverse

  const size_t nc2 = (size_t)pr.nc * pr.nc, nn = (size_t)n * n;
  // The determinant signs must read 0 unless this call's inverse finished.
  e = cudaMemset(d_sgn, 0, sizeof(int32_t) * 2);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffSiteSub, pr.site_sub, sizeof(int32_t) * nc2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffSiteAdd, add.data(), sizeof(int32_t) * nc2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffG0, g0.data(), sizeof(double) * table, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffProblem, &d, sizeof(d), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffWalker, &w, sizeof(w), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffSite, site.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffTau, tau.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kOffSpin, s.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    dca::launch_fresh_inverse(cfg, n, d_sgn, nullptr);
    e = cudaGetLastError();
  }
  int32_t sgn[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(sgn, d_sgn, sizeof(sgn), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && N_up) e = cudaMemcpy(N_up, w.N[0][0], sizeof(double) * nn, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && N_dn) e = cudaMemcpy(N_dn, w.N[0][1], sizeof(double) * nn, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(DCA_ERR_CUDA, cudaGetErrorString(e));
  if (sgn[0] == 0 || sgn[1] == 0) return fail(DCA_ERR_NUMERIC, "singular matrix");
  if (det_sign) *det_sign = sgn[0] * sgn[1];
  return DCA_OK;
}
