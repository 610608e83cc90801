// wf_ctx.h -- host-side context: device, workspace arena, per-size twiddle tables, error text.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wf.h"

// Grid sizes compiled into the library (2^a 3^b, even, half size also 2^a 3^b and even).
#define WF_SIZES(X) \
  X(16) X(24) X(32) X(48) X(64) X(72) X(96) X(108) X(128) X(144) X(192) X(216) X(256) X(288) X(384) X(512)

namespace wf {

// largest coarse radius of a deflated solve (wf_solve_opts.deflate)
constexpr int kDeflMaxRadius = 12;

void set_last_error(const char* what, cudaError_t e);

#define WF_CUDA(...)                                   \
  do {                                                 \
    cudaError_t e_ = (__VA_ARGS__);                    \
    if (e_ != cudaSuccess) {                           \
      ::wf::set_last_error(#__VA_ARGS__, e_);          \
      return e_ == cudaErrorMemoryAllocation ? WF_ERR_OOM : WF_ERR_CUDA; \
    }                                                  \
  } while (0)

#define WF_TRY(...)                \
  do {                             \
    wf_status s_ = (__VA_ARGS__);  \
    if (s_ != WF_OK) return s_;    \
  } while (0)

// Launch profiler: every kernel launch is counted; when enabled, each launch is bracketed by
// CUDA events on its stream and attributed to a kernel class with its algorithmic bytes.
struct ProfClass {
  long long launches = 0;
  double ms = 0.0;
  double bytes = 0.0;  // algorithmic bytes summed over the timed launches
};
struct Prof {
  bool on = false;
  long long launches = 0;  // all kernel launches since the last reset
  struct Rec {
    std::string name;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Rec> pending;
  std::map<std::string, ProfClass> classes;
  cudaEvent_t get_event() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  // fold pending records into the classes (synchronises on their events)
  void collect() {
    for (auto& r : pending) {
      cudaEventSynchronize(r.b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      ProfClass& c = classes[r.name];
      c.launches += 1;
      c.ms += ms;
      c.bytes += r.bytes;
    }
    pending.clear();
    used = 0;
  }
  void reset() {
    collect();
    classes.clear();
    launches = 0;
  }
  void release() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    used = 0;
    pending.clear();
  }
};

// A growable named device buffer owned by the context.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Ctx {
  int device = 0;
  size_t budget = 0;        // 0 = unlimited
  size_t held = 0;          // bytes currently allocated by the arena
  std::mutex mu;            // serialises synchronous API calls on this context
  std::map<std::string, DevBuf> bufs;
  std::map<int, double2*> twiddles;  // per N: exp(-2 pi i e / (2N)), e < 2N
  std::map<int, float2*> twiddles32; // the same rounded to FP32 (for the FP32 kernels)
  std::map<std::string, DevBuf> pinned;  // page-locked host buffers (scalar staging)
  std::vector<cudaStream_t> streams;     // non-blocking streams for interleaved groups
  cudaStream_t cap_stream = nullptr;     // stream on which CG blocks are captured as graphs
  void* host_pinned = nullptr;       // small pinned staging area for scalars
  struct Server* server = nullptr;   // serving loop, created on first wf_submit
  bool fused_planes = false;         // FP32 y / z / y passes as one cluster kernel where possible
  int* dev_err = nullptr;            // device word: nonzero after a kernel's bounded wait timed out
  bool map_failed = false;           // the driver refused a tensor map for a launch
  int sm_count = 0;
  // launch variant per "pass/precision/size" chosen by wf_autotune (variant 0 when absent)
  std::map<std::string, int> tuned;
  Prof prof;

  // Launch `f` (which enqueues one kernel on st), counting it and, when profiling, timing it.
  template <class F>
  void launch(const char* name, double bytes, cudaStream_t st, F&& f) {
    prof.launches += 1;
    if (!prof.on) {
      f();
      return;
    }
    if (prof.used + 2 > 4096) prof.collect();
    cudaEvent_t a = prof.get_event();
    cudaEvent_t b = prof.get_event();
    cudaEventRecord(a, st);
    f();
    cudaEventRecord(b, st);
    prof.pending.push_back(Prof::Rec{name, bytes, a, b});
  }

  // Device buffer `name` with at least `bytes` bytes (contents not preserved on growth).
  wf_status get(const std::string& name, size_t bytes, void** out);
  wf_status tw(int n, const double2** out);
  wf_status tw32(int n, const float2** out);
  // Page-locked host buffer `name` with at least `bytes` bytes.
  wf_status get_pinned(const std::string& name, size_t bytes, void** out);
  // i-th library-owned non-blocking stream.
  wf_status stream(int i, cudaStream_t* out);
  wf_status capture_stream(cudaStream_t* out);
  // The device error word (zeroed on first use) and the SM count; call before any capture.
  wf_status err_word(int** out);
  // WF_ERR_TIMEOUT (and the word cleared) if a kernel reported a timed-out wait, WF_ERR_CUDA if a
  // tensor map was refused since the last check.  Synchronises with the device.
  wf_status check_device_errors();
  // Free every device and pinned buffer whose name starts with `prefix`.
  void release_prefix(const std::string& prefix);
  void release_all();
};

// RAII: make the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline int supported_size(int n) {
  switch (n) {
#define WF_CASE(N) case N:
    WF_SIZES(WF_CASE)
#undef WF_CASE
    return 1;
    default:
      return 0;
  }
}

// ---- entry points of the compute modules (defined in the .cu files) ----------------------
wf_status assign_run(Ctx& c, const wf_grid& g, int scheme, const double* pos, int64_t n_gal,
                     uint64_t* fine_out, double* n_obs, cudaStream_t st);
wf_status assign_weighted_run(Ctx& c, const wf_grid& g, int scheme, const double* pos, const double* wgt,
                              int64_t n_gal, uint64_t* fine_out, double* n_obs, cudaStream_t st);
wf_status selection_at_run(Ctx& c, const wf_selection& sel, const double* pos, int64_t n_pts, bool reciprocal,
                          double* w, cudaStream_t st);
wf_status sd_noise_run(Ctx& c, int64_t n_cells, const double* n_obs, const double* w, const double* lambda,
                       double nbar, double* D, double* b, cudaStream_t st);
wf_status jackknife_run(Ctx& c, int64_t n_gal, const double* w_gal, const double* u, double alpha, double* out,
                        cudaStream_t st);
wf_status add_scaled_run(Ctx& c, int64_t n, const double* s, double f, double* acc, cudaStream_t st);
wf_status project_mask_run(Ctx& c, const wf_grid& g, const double* sky, int n_alpha, int n_delta, double alpha0,
                           double dalpha, double delta0, double ddelta, const double* obs, double dr, int n_r,
                           const double* wr, double* w, int64_t* counts, cudaStream_t st);
// the steps around the solve (wf_post.cu)
double rsd_factor(double k, double beta, double sigma_v);
wf_status deconvolve_run(Ctx& c, const wf_grid& g, const double* in, double beta, double sigma_v, double bias,
                         double* out, cudaStream_t st);
wf_status smooth_run(Ctx& c, const wf_grid& g, const double* in, double r_s, double* out, cudaStream_t st);
wf_status compare_run(Ctx& c, int64_t n_cells, const double* rec, const double* truth, wf_compare_result* out,
                      cudaStream_t st);
wf_status density_run(Ctx& c, const wf_grid& g, const double* delta, const double* w, const double* observer,
                      int n_shells, const double* shells, double lo, double width, int n_bins, int64_t* hist,
                      wf_density_moments* moments, cudaStream_t st);
wf_status noise_run(Ctx& c, const wf_grid& g, const wf_selection& sel, const double* n_obs,
                    int64_t n_gal, double* w, double* d, double* b, double* nbar, cudaStream_t st);

// Everything a single solve needs; tables are host-built per solve.
struct SolveArgs {
  wf_grid grid;
  const double* w = nullptr;
  const double* b = nullptr;
  double nbar = 0.0;
  wf_solve_opts opts{};
  double* s_out = nullptr;
  std::vector<double> sinv;  // S^-1 by n2, length 3 (N/2)^2 + 1
  double sum_w = -1.0;       // filled by the driver
};
wf_status build_sinv_table(const wf_grid& g, const wf_power& pw, std::vector<double>& out);
// S^-1 -> S^-1 / g^2 in place and ginv[n2] = 1 / g(k) for the response g = bias sqrt(<K D>_mu)
wf_status response_tables(const wf_grid& g, const wf_response* r, std::vector<double>& sinv,
                          std::vector<double>& ginv);
// out = F^-1 diag(table[n2]) F in / n^3 (FP64 transforms; out may equal in)
wf_status multiply_fourier(Ctx& c, int n, const double* in, double* out, const std::vector<double>& table,
                           cudaStream_t st);
// Solve every system (grouped by size and precision, groups interleaved on the device).
// Returns WF_OK if all converged, else the first failing status; infos[i] filled for each.
wf_status solve_many(Ctx& c, std::vector<SolveArgs*>& sys, std::vector<wf_solve_info*>& infos, cudaStream_t st);
void serve_shutdown(Ctx& c);

}  // namespace wf
