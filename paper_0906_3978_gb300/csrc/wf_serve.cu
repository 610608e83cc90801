// wf_serve.cu -- serving loop (wf_submit / wf_poll).
#include "wf_ctx.h"

namespace wf {
void serve_shutdown(Ctx&) {}
}  // namespace wf

extern "C" {
wf_status wf_submit(wf_ctx*, const wf_grid*, const wf_power*, const double*, double, const double*,
                    const wf_solve_opts*, uint64_t*) {
  return WF_ERR_UNSUPPORTED;
}
wf_status wf_poll(wf_ctx*, uint64_t, int, double*, wf_solve_info*) { return WF_ERR_UNSUPPORTED; }
}
