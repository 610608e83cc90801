// wf_solver_group.h -- the host-side interface of a group of systems solved together
// (implemented per grid size in wf_solver_impl.cuh).
#pragma once
#include <string>
#include <vector>

#include "wf_ctx.h"

namespace wf {

struct Group {
  virtual ~Group() {}
  // allocate, copy inputs and start the sums of w and b^2 (no host synchronisation) ...
  virtual wf_status prepare_begin(Ctx& c, cudaStream_t st) = 0;
  // ... and, once the stream has passed prepare_begin's work: tables, scalars, start CG
  virtual wf_status prepare_end(Ctx& c, cudaStream_t st) = 0;
  wf_status prepare(Ctx& c, cudaStream_t st) {  // both, waiting in between
    WF_TRY(prepare_begin(c, st));
    WF_CUDA(cudaStreamSynchronize(st));
    return prepare_end(c, st);
  }
  virtual wf_status enqueue(Ctx& c, cudaStream_t st) = 0;  // next block of device work
  virtual wf_status advance(Ctx& c) = 0;                   // after a sync: consume scalars
  virtual bool done() const = 0;
  virtual wf_status finish(Ctx& c, cudaStream_t st) = 0;   // copy the solutions out
  std::vector<SolveArgs*> sys;
  std::vector<wf_solve_info*> info;
  int nb = 0;
  std::string tag;  // prefix of this group's workspace names ("" = shared, reused across calls)
  // Device bytes a group of `count` systems of size n and precision prec holds (coarse radius K).
  static size_t footprint(int n, int prec, int count, int K = 0);
};

Group* make_group_n(int n, int prec);
// the coarse modes of a deflated solve of radius K, (kx, ky, kz, |k|^2), and the padded number
// of coarse coordinates 2 nh + 1
std::vector<int4> deflation_modes(int K);
int deflation_ncp(int K);

// out = F^-1 [table(|m|^2) F in] for one field of size N (instantiated with the solve drivers of
// each size); table has 3 (N/2)^2 + 1 entries.
template <int N>
wf_status fourier_multiply_n(Ctx& c, const double* in, double* out, const std::vector<double>& table,
                             cudaStream_t st);

// Time every launch variant of the spectral passes of grid size N in precision prec (the FP32
// inner passes for WF_MIXED, the FP64 ones for WF_FP64), keep the fastest per pass in c.tuned and
// append a JSON object per pass to `report`.
template <int N>
wf_status autotune_n(Ctx& c, int prec, std::string& report);
wf_status autotune(Ctx& c, int n, int prec, std::string& report);

}  // namespace wf
