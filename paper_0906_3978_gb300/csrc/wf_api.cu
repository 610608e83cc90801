// wf_api.cu -- the C ABI (include/wf.h): context, argument checks, dispatch to the kernels.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <map>
#include <memory>

#include "wf_ctx.h"

namespace wf {

struct Group;
template <int N>
Group* make_group(int prec);

static thread_local std::string g_last_error;

void set_last_error(const char* what, cudaError_t e) {
  g_last_error = e == cudaSuccess ? std::string(what) : std::string(what) + ": " + cudaGetErrorString(e);
}

wf_status Ctx::get(const std::string& name, size_t bytes, void** out) {
  if (bytes == 0) bytes = 16;
  DevBuf& b = bufs[name];
  if (b.ptr && b.bytes >= bytes) {
    *out = b.ptr;
    return WF_OK;
  }
  if (b.ptr) {
    cudaFree(b.ptr);
    held -= b.bytes;
    b.ptr = nullptr;
    b.bytes = 0;
  }
  if (budget && held + bytes > budget) return WF_ERR_OOM;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error("cudaMalloc", e);
    return WF_ERR_OOM;
  }
  b.ptr = p;
  b.bytes = bytes;
  held += bytes;
  *out = p;
  return WF_OK;
}

wf_status Ctx::err_word(int** out) {
  if (!dev_err) {
    void* p = nullptr;
    WF_TRY(get("dev_err", 64, &p));
    WF_CUDA(cudaMemset(p, 0, 64));
    dev_err = reinterpret_cast<int*>(p);
  }
  if (!sm_count) WF_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device));
  *out = dev_err;
  return WF_OK;
}

wf_status Ctx::check_device_errors() {
  if (map_failed) {
    map_failed = false;
    set_last_error("cuTensorMapEncodeTiled refused a spectrum map", cudaSuccess);
    return WF_ERR_CUDA;
  }
  if (!dev_err) return WF_OK;
  int h = 0;
  WF_CUDA(cudaMemcpy(&h, dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    WF_CUDA(cudaMemset(dev_err, 0, sizeof(int)));
    set_last_error("a kernel's wait for a bulk copy timed out", cudaSuccess);
    return WF_ERR_TIMEOUT;
  }
  return WF_OK;
}

wf_status Ctx::tw(int n, const double2** out) {
  auto it = twiddles.find(n);
  if (it != twiddles.end()) {
    *out = it->second;
    return WF_OK;
  }
  std::vector<double2> h((size_t)2 * n);
  const double pi = 3.14159265358979323846;
  for (int e = 0; e < 2 * n; ++e) {
    const double ang = 2.0 * pi * (double)e / (2.0 * n);
    h[e] = make_double2(std::cos(ang), -std::sin(ang));
  }
  double2* d = nullptr;
  WF_CUDA(cudaMalloc(&d, h.size() * sizeof(double2)));
  WF_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
  twiddles[n] = d;
  *out = d;
  return WF_OK;
}

wf_status Ctx::tw32(int n, const float2** out) {
  auto it = twiddles32.find(n);
  if (it != twiddles32.end()) {
    *out = it->second;
    return WF_OK;
  }
  std::vector<float2> h((size_t)2 * n);
  const double pi = 3.14159265358979323846;
  for (int e = 0; e < 2 * n; ++e) {
    const double ang = 2.0 * pi * (double)e / (2.0 * n);
    h[e] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
  }
  float2* d = nullptr;
  WF_CUDA(cudaMalloc(&d, h.size() * sizeof(float2)));
  WF_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice));
  twiddles32[n] = d;
  *out = d;
  return WF_OK;
}

wf_status Ctx::get_pinned(const std::string& name, size_t bytes, void** out) {
  if (bytes == 0) bytes = 16;
  DevBuf& b = pinned[name];
  if (b.ptr && b.bytes >= bytes) {
    *out = b.ptr;
    return WF_OK;
  }
  if (b.ptr) {
    cudaFreeHost(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  WF_CUDA(cudaMallocHost(&b.ptr, bytes));
  b.bytes = bytes;
  *out = b.ptr;
  return WF_OK;
}

wf_status Ctx::stream(int i, cudaStream_t* out) {
  while ((int)streams.size() <= i) {
    cudaStream_t s;
    WF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    streams.push_back(s);
  }
  *out = streams[i];
  return WF_OK;
}

wf_status Ctx::capture_stream(cudaStream_t* out) {
  if (!cap_stream) WF_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
  *out = cap_stream;
  return WF_OK;
}

void Ctx::release_prefix(const std::string& prefix) {
  for (auto it = bufs.begin(); it != bufs.end();) {
    if (it->first.compare(0, prefix.size(), prefix) == 0) {
      if (it->second.ptr) cudaFree(it->second.ptr);
      held -= it->second.bytes;
      it = bufs.erase(it);
    } else {
      ++it;
    }
  }
  for (auto it = pinned.begin(); it != pinned.end();) {
    if (it->first.compare(0, prefix.size(), prefix) == 0) {
      if (it->second.ptr) cudaFreeHost(it->second.ptr);
      it = pinned.erase(it);
    } else {
      ++it;
    }
  }
}

void Ctx::release_all() {
  for (auto& kv : bufs)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  bufs.clear();
  dev_err = nullptr;
  held = 0;
  for (auto& kv : twiddles) cudaFree(kv.second);
  twiddles.clear();
  for (auto& kv : twiddles32) cudaFree(kv.second);
  twiddles32.clear();
  for (auto& kv : pinned)
    if (kv.second.ptr) cudaFreeHost(kv.second.ptr);
  pinned.clear();
  for (auto s : streams) cudaStreamDestroy(s);
  streams.clear();
  if (cap_stream) cudaStreamDestroy(cap_stream);
  cap_stream = nullptr;
}

// P(k) by log-log linear interpolation in the table (end segments extrapolated);
// S^-1[n2] = dV / P(2 pi sqrt(n2) / L), S^-1[0] = 0.
wf_status build_sinv_table(const wf_grid& g, const wf_power& pw, std::vector<double>& out) {
  if (!pw.k || !pw.p || pw.n < 2) return WF_ERR_ARG;
  for (int i = 0; i < pw.n; ++i)
    if (!(pw.k[i] > 0.0) || !(pw.p[i] > 0.0) || !std::isfinite(pw.k[i]) || !std::isfinite(pw.p[i]) ||
        (i > 0 && !(pw.k[i] > pw.k[i - 1])))
      return WF_ERR_ARG;
  const long half = g.n / 2, len = 3 * half * half + 1;
  const double H = g.box / (double)g.n, dV = H * H * H;
  const double kf = 2.0 * 3.14159265358979323846 / g.box;
  std::vector<double> lk(pw.n), lp(pw.n);
  for (int i = 0; i < pw.n; ++i) {
    lk[i] = std::log(pw.k[i]);
    lp[i] = std::log(pw.p[i]);
  }
  out.assign((size_t)len, 0.0);
  int seg = 0;
  for (long n2 = 1; n2 < len; ++n2) {
    const double k = kf * std::sqrt((double)n2);
    while (seg < pw.n - 2 && k > pw.k[seg + 1]) ++seg;  // k grows with n2
    const double t = (std::log(k) - lk[seg]) / (lk[seg + 1] - lk[seg]);
    const double p = std::exp(lp[seg] + t * (lp[seg + 1] - lp[seg]));
    out[(size_t)n2] = dV / p;
    if (!(out[(size_t)n2] > 0.0) || !std::isfinite(out[(size_t)n2])) return WF_ERR_ARG;
  }
  return WF_OK;
}

}  // namespace wf
#include "wf_solver_group.h"
namespace wf {

Group* make_group_n(int n, int prec) {
  switch (n) {
#define WF_CASE(N) \
  case N:          \
    return make_group<N>(prec);
    WF_SIZES(WF_CASE)
#undef WF_CASE
    default:
      return nullptr;
  }
}

wf_status autotune(Ctx& c, int n, int prec, std::string& report) {
  switch (n) {
#define WF_CASE(N) \
  case N:          \
    return autotune_n<N>(c, prec, report);
    WF_SIZES(WF_CASE)
#undef WF_CASE
    default:
      return WF_ERR_UNSUPPORTED;
  }
}

// The coarse radius deflate = -1 picks: the fastest of a sweep of the radii at each size on the
// 512^3 workload's recipe and cell size (n 64: 3, <= 128: 4, <= 192: 6, <= 256: 8, <= 384: 10,
// above: 12); none below 64, where the iteration counts are small and the extra launches cost more.
int auto_deflate(int n) {
  if (n < 64) return 0;
  if (n == 64) return 3;
  if (n <= 128) return 4;
  if (n <= 192) return 6;
  if (n <= 256) return 8;
  if (n <= 384) return 10;
  return 12;
}

// Coarse modes of radius K: one of each +-k pair, k != 0 (kz > 0, or kz = 0 with ky > 0, or
// kz = ky = 0 with kx > 0), as (kx, ky, kz, |k|^2), in the order kz, ky, kx.
std::vector<int4> deflation_modes(int K) {
  std::vector<int4> m;
  for (int kz = 0; kz <= K; ++kz)
    for (int ky = -K; ky <= K; ++ky)
      for (int kx = -K; kx <= K; ++kx) {
        const int n2 = kx * kx + ky * ky + kz * kz;
        if (n2 > K * K || n2 == 0) continue;
        if (kz > 0 || ky > 0 || (ky == 0 && kx > 0)) m.push_back(make_int4(kx, ky, kz, n2));
      }
  return m;
}
int deflation_ncp(int K) {
  const int nc = 2 * (int)deflation_modes(K).size() + 1;
  return (nc + 127) / 128 * 128;  // whole 128 x 128 tiles of the Gauss-Jordan update
}

// Device bytes of a group (the buffers GroupFP64 / GroupMixed allocate, tables excluded), with the
// coarse-space buffers of a deflated group (K > 0).
size_t Group::footprint(int n, int prec, int count, int K) {
  const double V = (double)n * n * n, spec = V / 2;
  double per = prec == WF_MIXED ? 5 * spec * 8 + 2 * spec * 16 + 4 * V + 4 * 8 * V : 6 * spec * 16 + 5 * 8 * V;
  if (K > 0) {
    const double ncp = deflation_ncp(K), C = 4.0 * K + 1;
    per += 4 * ncp * ncp + 2 * 4 * 64 * ncp + 8 * ncp + 8 * (double)n * n * (K + 1) +
           8 * (2.0 * K + 1) * (K + 1) * n + 8 * C * C * C + 24 * ncp + 8 * 64 * 64 + 4.0 * (3 * (n / 2) * (n / 2) + 1);
  }
  return (size_t)(per * count) + (size_t)count * (3 * (n / 2) * (n / 2) + 1) * 24 + (64u << 10);
}

wf_status solve_many(Ctx& c, std::vector<SolveArgs*>& sys, std::vector<wf_solve_info*>& infos, cudaStream_t st) {
  std::map<std::tuple<int, int, int>, std::unique_ptr<Group>> groups;
  for (size_t i = 0; i < sys.size(); ++i) {
    const auto key = std::make_tuple(sys[i]->grid.n, (int)sys[i]->opts.prec, sys[i]->opts.deflate);
    auto& g = groups[key];
    if (!g) {
      g.reset(make_group_n(std::get<0>(key), std::get<1>(key)));
      if (!g) return WF_ERR_UNSUPPORTED;
    }
    g->sys.push_back(sys[i]);
    g->info.push_back(infos[i]);
  }
  // one stream per group (the caller's stream when there is a single group)
  std::vector<Group*> gl;
  std::vector<cudaStream_t> gs;
  cudaEvent_t ev;
  WF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  WF_CUDA(cudaEventRecord(ev, st));
  int k = 0;
  for (auto& kv : groups) {
    cudaStream_t s = st;
    if (groups.size() > 1) {
      WF_TRY(c.stream(k, &s));
      WF_CUDA(cudaStreamWaitEvent(s, ev, 0));
    }
    gl.push_back(kv.second.get());
    gs.push_back(s);
    ++k;
  }
  int* err = nullptr;
  WF_TRY(c.err_word(&err));
  wf_status status = WF_OK;
  // start every group's preparation, then finish each one as its stream gets there
  for (size_t i = 0; i < gl.size() && status == WF_OK; ++i) status = gl[i]->prepare_begin(c, gs[i]);
  for (size_t i = 0; i < gl.size() && status == WF_OK; ++i) {
    WF_CUDA(cudaStreamSynchronize(gs[i]));
    status = gl[i]->prepare_end(c, gs[i]);
  }
  // Each group alternates a block of device work (ending with an event) and the host step that
  // reads its scalars.  A group whose block has finished takes its host step and starts its next
  // block at once, without waiting for the slower groups.
  std::vector<cudaEvent_t> evs(gl.size(), nullptr);
  std::vector<char> inflight(gl.size(), 0);
  for (size_t i = 0; i < gl.size() && status == WF_OK; ++i)
    if (cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming) != cudaSuccess) status = WF_ERR_CUDA;
  while (status == WF_OK) {
    bool any = false, progressed = false;
    int running = -1, n_running = 0;
    for (size_t i = 0; i < gl.size() && status == WF_OK; ++i) {
      if (gl[i]->done()) continue;
      any = true;
      if (inflight[i]) {
        const cudaError_t q = cudaEventQuery(evs[i]);
        if (q == cudaErrorNotReady) {
          running = (int)i;
          ++n_running;
          continue;
        }
        if (q != cudaSuccess) {
          set_last_error("CG block", q);
          status = WF_ERR_CUDA;
          break;
        }
        inflight[i] = 0;
        status = gl[i]->advance(c);
        progressed = true;
        if (status != WF_OK || gl[i]->done()) continue;
      }
      status = gl[i]->enqueue(c, gs[i]);
      if (status == WF_OK && cudaEventRecord(evs[i], gs[i]) != cudaSuccess) status = WF_ERR_CUDA;
      inflight[i] = 1;
      progressed = true;
    }
    if (!any || status != WF_OK) break;
    if (!progressed) {
      if (n_running == 1) cudaEventSynchronize(evs[running]);  // a single group: just wait for it
      else std::this_thread::yield();
    }
  }
  for (auto e : evs)
    if (e) cudaEventDestroy(e);
  for (size_t i = 0; i < gl.size() && status == WF_OK; ++i) {
    status = gl[i]->finish(c, gs[i]);
    if (status == WF_OK && gs[i] != st) {
      WF_CUDA(cudaEventRecord(ev, gs[i]));
      WF_CUDA(cudaStreamWaitEvent(st, ev, 0));
    }
  }
  WF_CUDA(cudaStreamSynchronize(st));
  cudaEventDestroy(ev);
  if (status != WF_OK) return status;
  WF_TRY(c.check_device_errors());
  for (auto* inf : infos)
    if (inf && inf->status != WF_OK) return inf->status;
  return WF_OK;
}

static wf_status check_grid(const wf_grid* g) {
  if (!g) return WF_ERR_ARG;
  if (!supported_size(g->n)) return WF_ERR_UNSUPPORTED;
  if (!(g->box > 0.0) || !std::isfinite(g->box)) return WF_ERR_ARG;
  return WF_OK;
}

wf_status prepare_solve(const wf_grid* grid, const wf_power* power, const double* w, double nbar,
                        const double* b, const wf_solve_opts* opts, double* s_out, SolveArgs& a) {
  WF_TRY(check_grid(grid));
  if (!power || !w || !b || !s_out || !opts) return WF_ERR_ARG;
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return WF_ERR_ARG;
  if (!(opts->tol > 0.0) || opts->max_iter <= 0 || (opts->prec != WF_FP64 && opts->prec != WF_MIXED))
    return WF_ERR_ARG;
  if (opts->deflate != 0 && opts->deflate != -1 &&
      (opts->prec != WF_MIXED || opts->deflate < 1 || opts->deflate > kDeflMaxRadius || 4 * opts->deflate >= grid->n)) {
    set_last_error("deflate: a coarse radius in [1, 12] with 4 K < n, for WF_MIXED solves only", cudaSuccess);
    return WF_ERR_ARG;
  }
  a.grid = *grid;
  a.w = w;
  a.b = b;
  a.nbar = nbar;
  a.opts = *opts;
  if (a.opts.deflate == -1) a.opts.deflate = opts->prec == WF_MIXED ? auto_deflate(grid->n) : 0;
  a.s_out = s_out;
  return build_sinv_table(*grid, *power, a.sinv);
}

}  // namespace wf

using namespace wf;

extern "C" {

int wf_supported_size(int n) { return supported_size(n); }

int wf_deflate_radius(int n, wf_precision prec) { return prec == WF_MIXED ? auto_deflate(n) : 0; }

const char* wf_last_error(void) { return g_last_error.c_str(); }

const char* wf_status_string(wf_status s) {
  switch (s) {
    case WF_OK: return "ok";
    case WF_PENDING: return "pending";
    case WF_ERR_ARG: return "invalid argument";
    case WF_ERR_OOM: return "out of device memory or over the HBM budget";
    case WF_ERR_CUDA: return "CUDA error";
    case WF_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case WF_ERR_BREAKDOWN: return "CG breakdown";
    case WF_ERR_TIMEOUT: return "timeout";
    case WF_ERR_OVERFLOW: return "fine-grid cell overflow";
    case WF_ERR_BUSY: return "queue full";
    case WF_ERR_UNSUPPORTED: return "grid size not supported";
  }
  return "unknown status";
}

wf_status wf_create(wf_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return WF_ERR_ARG;
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) {
    set_last_error("cudaGetDeviceCount", e);
    return WF_ERR_CUDA;
  }
  if (device < 0 || device >= count) return WF_ERR_ARG;
  Ctx* c = new Ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  DeviceGuard g(device);
  e = cudaMallocHost(&c->host_pinned, 4096);
  if (e != cudaSuccess) {
    set_last_error("cudaMallocHost", e);
    delete c;
    return WF_ERR_CUDA;
  }
  *out = reinterpret_cast<wf_ctx*>(c);
  return WF_OK;
}

wf_status wf_destroy(wf_ctx* ctx) {
  if (!ctx) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  {
    DeviceGuard g(c->device);
    serve_shutdown(*c);
    cudaDeviceSynchronize();
    c->prof.reset();
    c->prof.release();
    c->release_all();
    if (c->host_pinned) cudaFreeHost(c->host_pinned);
  }
  delete c;
  return WF_OK;
}

wf_status wf_grid_assign(wf_ctx* ctx, const wf_grid* grid, wf_scheme scheme, const double* pos, int64_t n_gal,
                         uint64_t* fine_out, double* n_obs, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return assign_run(*c, *grid, (int)scheme, pos, n_gal, fine_out, n_obs, (cudaStream_t)stream);
}

wf_status wf_build_noise(wf_ctx* ctx, const wf_grid* grid, const wf_selection* sel, const double* n_obs,
                         int64_t n_gal, double* w, double* d, double* b, double* nbar, void* stream) {
  if (!ctx || !sel) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return noise_run(*c, *grid, *sel, n_obs, n_gal, w, d, b, nbar, (cudaStream_t)stream);
}

wf_status wf_solve(wf_ctx* ctx, const wf_grid* grid, const wf_power* power, const double* w, double nbar,
                   const double* b, const wf_solve_opts* opts, double* s_out, wf_solve_info* info, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  SolveArgs a;
  wf_status s = prepare_solve(grid, power, w, nbar, b, opts, s_out, a);
  if (s != WF_OK) {
    if (info) info->status = s;
    return s;
  }
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  wf_solve_info tmp{};
  std::vector<SolveArgs*> sys{&a};
  std::vector<wf_solve_info*> infos{info ? info : &tmp};
  s = solve_many(*c, sys, infos, (cudaStream_t)stream);
  if (info) info->status = s;
  return s;
}

wf_status wf_solve_response(wf_ctx* ctx, const wf_grid* grid, const wf_power* power, const wf_response* response,
                            const double* w, double nbar, const double* b, const wf_solve_opts* opts,
                            double* s_out, wf_solve_info* info, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  SolveArgs a;
  wf_status s = prepare_solve(grid, power, w, nbar, b, opts, s_out, a);
  // s_out is deconvolved in place after the solve: it must not share a byte with w or b
  if (s == WF_OK) {
    const size_t bytes = sizeof(double) * (size_t)grid->n * grid->n * grid->n;
    const auto overlaps = [bytes](const void* p, const void* q) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(p), c = reinterpret_cast<uintptr_t>(q);
      return a < c + bytes && c < a + bytes;
    };
    if (overlaps(s_out, w) || overlaps(s_out, b)) {
      set_last_error("wf_solve_response: s_out overlaps w or b", cudaSuccess);
      s = WF_ERR_ARG;
    }
  }
  std::vector<double> ginv;
  if (s == WF_OK) s = response_tables(*grid, response, a.sinv, ginv);
  if (s != WF_OK) {
    if (info) info->status = s;
    return s;
  }
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  wf_solve_info tmp{};
  std::vector<SolveArgs*> sys{&a};
  wf_solve_info* inf = info ? info : &tmp;
  std::vector<wf_solve_info*> infos{inf};
  s = solve_many(*c, sys, infos, (cudaStream_t)stream);
  // s_m = G^-1 s_g; also on a non-converged exit, so that s_out always holds the matter field
  const wf_status sd = multiply_fourier(*c, grid->n, s_out, s_out, ginv, (cudaStream_t)stream);
  if (s == WF_OK) s = sd;
  inf->status = s;
  return s;
}

wf_status wf_jackknife_solve(wf_ctx* ctx, const wf_grid* grid, wf_scheme scheme, const wf_power* power,
                             const double* pos, int64_t n_gal, const double* w_gal, const double* u, int n_sub,
                             double alpha, const double* n_obs, const double* w, double nbar,
                             const wf_solve_opts* opts, double* s_mean, wf_solve_info* infos, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  if (!power || !pos || !w_gal || !u || !n_obs || !w || !s_mean || !opts || n_gal <= 0 || n_sub <= 0 ||
      !(alpha > 0.0) || !(alpha <= 1.0) || !(nbar > 0.0) || !std::isfinite(nbar))
    return WF_ERR_ARG;
  if (!(opts->tol > 0.0) || opts->max_iter <= 0 || (opts->prec != WF_FP64 && opts->prec != WF_MIXED))
    return WF_ERR_ARG;
  if (opts->deflate != 0 && opts->deflate != -1 &&
      (opts->prec != WF_MIXED || opts->deflate < 1 || opts->deflate > kDeflMaxRadius || 4 * opts->deflate >= grid->n)) {
    set_last_error("deflate: a coarse radius in [1, 12] with 4 K < n, for WF_MIXED solves only", cudaSuccess);
    return WF_ERR_ARG;
  }
  if (infos) std::memset(infos, 0, (size_t)n_sub * sizeof(*infos));
  std::vector<double> sinv;
  WF_TRY(build_sinv_table(*grid, *power, sinv));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard dg(c->device);
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t V = (int64_t)grid->n * grid->n * grid->n;
  const int chunk = n_sub < 8 ? n_sub : 8;  // subsample systems solved together
  double *masses, *lam, *db, *sj;
  WF_TRY(c->get("jk_masses", (size_t)n_gal * sizeof(double), (void**)&masses));
  WF_TRY(c->get("jk_lambda", (size_t)V * sizeof(double), (void**)&lam));
  WF_TRY(c->get("jk_db", (size_t)chunk * 2 * V * sizeof(double), (void**)&db));
  WF_TRY(c->get("jk_s", (size_t)chunk * V * sizeof(double), (void**)&sj));
  WF_CUDA(cudaMemsetAsync(s_mean, 0, (size_t)V * sizeof(double), st));
  wf_status first_bad = WF_OK;
  for (int j0 = 0; j0 < n_sub; j0 += chunk) {
    const int m = std::min(chunk, n_sub - j0);
    std::vector<SolveArgs> args((size_t)m);
    std::vector<wf_solve_info> tmp((size_t)m);
    std::vector<SolveArgs*> sys;
    std::vector<wf_solve_info*> inf;
    for (int q = 0; q < m; ++q) {
      const int j = j0 + q;
      double* D = db + (size_t)(2 * q) * V;
      double* b = D + V;
      // subsample j (Eq. eq:selfunc), its low-passed grid N'' as lambda, the noise of Eq. eq:noisecov
      WF_TRY(jackknife_run(*c, n_gal, w_gal, u + (size_t)j * n_gal, alpha, masses, st));
      WF_TRY(assign_weighted_run(*c, *grid, (int)scheme, pos, masses, n_gal, nullptr, lam, st));
      WF_TRY(sd_noise_run(*c, V, n_obs, w, lam, nbar, D, b, st));
      SolveArgs& a = args[(size_t)q];
      a.grid = *grid;
      a.grid.supersample = 1;
      a.w = D;
      a.b = b;
      a.nbar = 1.0;
      a.opts = *opts;
      // -1: the radius by grid size, as for wf_solve.  Subsamples whose deflated inner solves break
      // down or stall (a few percent of sparse ones) continue as plain CG (wf_solver_impl.cuh)
      if (a.opts.deflate == -1) a.opts.deflate = opts->prec == WF_MIXED ? auto_deflate(grid->n) : 0;
      a.s_out = sj + (size_t)q * V;
      a.sinv = sinv;
      sys.push_back(&a);
      inf.push_back(infos ? infos + j : &tmp[(size_t)q]);
    }
    const wf_status s = solve_many(*c, sys, inf, st);
    if (s != WF_OK && first_bad == WF_OK) first_bad = s;
    for (int q = 0; q < m; ++q) WF_TRY(add_scaled_run(*c, V, sj + (size_t)q * V, 1.0 / n_sub, s_mean, st));
  }
  return first_bad;
}

wf_status wf_project_mask(wf_ctx* ctx, const wf_grid* grid, const double* sky, int n_alpha, int n_delta,
                          double alpha0, double dalpha, double delta0, double ddelta, const double* observer,
                          double dr, int n_r, const double* wr, double* w, int64_t* counts, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return project_mask_run(*c, *grid, sky, n_alpha, n_delta, alpha0, dalpha, delta0, ddelta, observer, dr, n_r, wr,
                          w, counts, (cudaStream_t)stream);
}

wf_status wf_sd_noise(wf_ctx* ctx, int64_t n_cells, const double* n_obs, const double* w, const double* lambda,
                      double nbar, double* D, double* b, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return sd_noise_run(*c, n_cells, n_obs, w, lambda, nbar, D, b, (cudaStream_t)stream);
}

wf_status wf_jackknife_masses(wf_ctx* ctx, int64_t n_gal, const double* w_gal, const double* u, double alpha,
                              double* out, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return jackknife_run(*c, n_gal, w_gal, u, alpha, out, (cudaStream_t)stream);
}

wf_status wf_selection_eval(wf_ctx* ctx, const wf_selection* sel, const double* pos, int64_t n_pts,
                            int reciprocal, double* w, void* stream) {
  if (!ctx || !sel) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return selection_at_run(*c, *sel, pos, n_pts, reciprocal != 0, w, (cudaStream_t)stream);
}

wf_status wf_grid_assign_weighted(wf_ctx* ctx, const wf_grid* grid, wf_scheme scheme, const double* pos,
                                  const double* wgt, int64_t n_gal, uint64_t* fine_out, double* n_obs,
                                  void* stream) {
  if (!ctx) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return assign_weighted_run(*c, *grid, (int)scheme, pos, wgt, n_gal, fine_out, n_obs, (cudaStream_t)stream);
}

wf_status wf_rsd_factor(int64_t n_k, const double* k, double beta, double sigma_v, double* out) {
  if (n_k < 0 || (n_k > 0 && (!k || !out)) || !std::isfinite(beta) || !(sigma_v >= 0.0) || !std::isfinite(sigma_v))
    return WF_ERR_ARG;
  for (int64_t i = 0; i < n_k; ++i) {
    if (!(k[i] >= 0.0) || !std::isfinite(k[i])) return WF_ERR_ARG;
    out[i] = rsd_factor(k[i], beta, sigma_v);
  }
  return WF_OK;
}

wf_status wf_deconvolve(wf_ctx* ctx, const wf_grid* grid, const double* in, double beta, double sigma_v,
                        double bias, double* out, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return deconvolve_run(*c, *grid, in, beta, sigma_v, bias, out, (cudaStream_t)stream);
}

wf_status wf_smooth(wf_ctx* ctx, const wf_grid* grid, const double* in, double r_s, double* out, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return smooth_run(*c, *grid, in, r_s, out, (cudaStream_t)stream);
}

wf_status wf_compare(wf_ctx* ctx, int64_t n_cells, const double* rec, const double* truth, wf_compare_result* out,
                     void* stream) {
  if (!ctx) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return compare_run(*c, n_cells, rec, truth, out, (cudaStream_t)stream);
}

wf_status wf_density_stats(wf_ctx* ctx, const wf_grid* grid, const double* delta, const double* w,
                           const double* observer, int n_shells, const double* shells, double lo, double width,
                           int n_bins, int64_t* hist, wf_density_moments* moments, void* stream) {
  if (!ctx) return WF_ERR_ARG;
  WF_TRY(check_grid(grid));
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return density_run(*c, *grid, delta, w, observer, n_shells, shells, lo, width, n_bins, hist, moments,
                     (cudaStream_t)stream);
}

static wf_status copy_text(const std::string& t, char* out, int len) {
  if (!out || len <= 0) return WF_ERR_ARG;
  if ((int)t.size() + 1 > len) {
    set_last_error("output buffer too small for the JSON text", cudaSuccess);
    return WF_ERR_ARG;
  }
  std::memcpy(out, t.c_str(), t.size() + 1);
  return WF_OK;
}

wf_status wf_autotune(wf_ctx* ctx, int n, wf_precision prec, char* report, int report_len) {
  if (!ctx || (prec != WF_FP64 && prec != WF_MIXED)) return WF_ERR_ARG;
  if (!supported_size(n)) return WF_ERR_UNSUPPORTED;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  std::string rep = "[";
  WF_TRY(autotune(*c, n, (int)prec, rep));
  rep += "]";
  return report ? copy_text(rep, report, report_len) : WF_OK;
}

wf_status wf_tune_get(wf_ctx* ctx, char* json, int len) {
  if (!ctx) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  std::string t = "{";
  bool first = true;
  for (const auto& kv : c->tuned) {
    t += (first ? "\"" : ", \"") + kv.first + "\": " + std::to_string(kv.second);
    first = false;
  }
  t += "}";
  return copy_text(t, json, len);
}

// Reads {"pass/prec/n": variant, ...}: every quoted key followed by ':' and an integer.
wf_status wf_tune_set(wf_ctx* ctx, const char* json) {
  if (!ctx || !json) return WF_ERR_ARG;
  std::map<std::string, int> parsed;
  const char* p = json;
  while ((p = std::strchr(p, '"'))) {
    const char* q = std::strchr(p + 1, '"');
    if (!q) return WF_ERR_ARG;
    std::string key(p + 1, q);
    const char* r = q + 1;
    while (*r == ' ' || *r == '\t' || *r == '\n') ++r;
    if (*r != ':') return WF_ERR_ARG;
    char* end = nullptr;
    const long v = std::strtol(r + 1, &end, 10);
    if (end == r + 1 || v < 0 || v > 1000) return WF_ERR_ARG;
    parsed[key] = (int)v;
    p = end;
  }
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  for (const auto& kv : parsed) c->tuned[kv.first] = kv.second;
  return WF_OK;
}

wf_status wf_set_fused_planes(wf_ctx* ctx, int on) {
  if (!ctx) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  c->fused_planes = on != 0;
  return WF_OK;
}

wf_status wf_profile(wf_ctx* ctx, int enable) {
  if (!ctx) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  c->prof.reset();
  c->prof.on = enable != 0;
  return WF_OK;
}

wf_status wf_profile_read(wf_ctx* ctx, int64_t* launches, int* n_classes) {
  if (!ctx || !launches || !n_classes) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  c->prof.collect();
  *launches = c->prof.launches;
  *n_classes = (int)c->prof.classes.size();
  return WF_OK;
}

wf_status wf_profile_class(wf_ctx* ctx, int i, char* name, int name_len, int64_t* launches, double* total_ms,
                           double* bytes) {
  if (!ctx || !name || name_len <= 0 || !launches || !total_ms || !bytes) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  if (i < 0 || i >= (int)c->prof.classes.size()) return WF_ERR_ARG;
  auto it = c->prof.classes.begin();
  std::advance(it, i);
  std::snprintf(name, (size_t)name_len, "%s", it->first.c_str());
  *launches = it->second.launches;
  *total_ms = it->second.ms;
  *bytes = it->second.bytes;
  return WF_OK;
}

wf_status wf_solve_batch(wf_ctx* ctx, int count, const wf_grid* grids, const wf_power* powers, const double* const* w,
                         const double* nbar, const double* const* b, const wf_solve_opts* opts, double* const* s_out,
                         wf_solve_info* infos, void* stream) {
  if (!ctx || count < 0 || (count > 0 && (!grids || !powers || !w || !nbar || !b || !opts || !s_out)))
    return WF_ERR_ARG;
  if (count == 0) return WF_OK;
  std::vector<SolveArgs> args((size_t)count);
  std::vector<wf_solve_info> tmp((size_t)count);
  std::vector<SolveArgs*> sys;
  std::vector<wf_solve_info*> inf;
  for (int i = 0; i < count; ++i) {
    wf_solve_info* pi = infos ? infos + i : &tmp[i];
    std::memset(pi, 0, sizeof(*pi));
    wf_status s = prepare_solve(grids + i, powers + i, w[i], nbar[i], b[i], opts + i, s_out[i], args[i]);
    if (s != WF_OK) {
      pi->status = s;
      return s;
    }
    sys.push_back(&args[i]);
    inf.push_back(pi);
  }
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return solve_many(*c, sys, inf, (cudaStream_t)stream);
}

}  // extern "C"
