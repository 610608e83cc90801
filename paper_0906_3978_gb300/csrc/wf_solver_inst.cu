// wf_solver_inst.cu -- instantiates the solve drivers (and the Fourier-multiplier pass) for one grid size (compiled once per
// size with -DWF_N=<n>, so the sizes build in parallel).
#include "wf_solver_impl.cuh"

#ifndef WF_N
#error "compile with -DWF_N=<grid size>"
#endif

namespace wf {
template Group* make_group<WF_N>(int prec);
template wf_status fourier_multiply_n<WF_N>(Ctx& c, const double* in, double* out, const std::vector<double>& table,
                                            cudaStream_t st);
template wf_status autotune_n<WF_N>(Ctx& c, int prec, std::string& report);
}
