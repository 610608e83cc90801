// wf_serve.cu -- serving loop behind wf_submit / wf_poll: continuous batching of Wiener solves.
//
// A scheduler thread per context owns a FIFO of submitted requests and a list of resident
// groups (systems of one grid size and precision advanced together by the batched kernels).
// Each group moves through three states, each a piece of device work on the group's own stream
// followed by an event: preparation (input copies, sums), running (blocks of CG iterations, one
// host step between blocks), finishing (the solutions' copy to the requests' host buffers).  The
// scheduler loop (1) admits queued requests in arrival order while the device footprint of the
// resident systems plus theirs fits the HBM budget and fewer than kMaxResident systems are
// resident, forming new groups and starting their preparation; (2) polls every resident group's
// event and, for each group whose work has finished, takes its next step at once -- a small
// group does not wait for a 384^3 block of another group, and admissions are checked between
// steps; (3) releases finished groups and wakes the pollers.  Request buffers are page-locked
// (up to kPinnedCap bytes in total) so that the copies in and out are asynchronous.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <tuple>

#include "wf_ctx.h"
#include "wf_solver_group.h"

namespace wf {

wf_status prepare_solve(const wf_grid* grid, const wf_power* power, const double* w, double nbar,
                        const double* b, const wf_solve_opts* opts, double* s_out, SolveArgs& a);

namespace {
constexpr int kMaxResident = 160;
constexpr size_t kMaxQueued = 4096;
constexpr int kFirstStream = 8;  // library streams 0..7 belong to wf_solve_batch
constexpr size_t kPinnedCap = (size_t)16 << 30;  // page-locked request buffers, all requests together
using Clock = std::chrono::steady_clock;
std::atomic<size_t> g_pinned{0};
}  // namespace

// Host copy of a request's w, b and solution s (3 V doubles), page-locked while the total stays
// under kPinnedCap, else ordinary memory (its copies then block the scheduler for their duration).
struct HostBuf {
  double* p = nullptr;
  size_t bytes = 0;
  bool pinned = false;
  std::vector<double> heap;
  bool alloc(size_t n) {
    bytes = n * sizeof(double);
    if (g_pinned.fetch_add(bytes) + bytes <= kPinnedCap &&
        cudaHostAlloc((void**)&p, bytes, cudaHostAllocDefault) == cudaSuccess) {
      pinned = true;
      return true;
    }
    g_pinned.fetch_sub(bytes);
    cudaGetLastError();
    heap.assign(n, 0.0);
    p = heap.data();
    return true;
  }
  ~HostBuf() {
    if (pinned) {
      cudaFreeHost(p);
      g_pinned.fetch_sub(bytes);
    }
  }
};

struct Request {
  uint64_t id = 0;
  HostBuf buf;                 // [w | b | s], V doubles each; s receives the solution
  double *w = nullptr, *b = nullptr, *s = nullptr;
  size_t V = 0;
  std::vector<double> k, p;
  SolveArgs args;
  wf_solve_info info{};
  wf_status status = WF_PENDING;
  Clock::time_point t_submit;
  size_t footprint = 0;
};

enum { RG_PREP = 0, RG_RUN = 1, RG_FIN = 2 };

struct ResidentGroup {
  std::unique_ptr<Group> g;
  std::vector<std::shared_ptr<Request>> reqs;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;   // end of the group's latest piece of device work
  int stream_idx = 0;
  size_t footprint = 0;
  int state = RG_PREP;
  bool inflight = false;
};

struct Server {
  Ctx* ctx = nullptr;
  std::thread th;
  std::mutex mu;                  // guards queue, requests, stop
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> requests;
  std::vector<ResidentGroup> resident;  // touched by the scheduler thread only
  std::vector<int> free_streams;
  uint64_t next_id = 1;
  uint64_t next_group = 1;
  int next_stream = kFirstStream;
  bool stop = false;
  size_t budget = 0, used = 0;
  int resident_systems = 0;

  void run();
  void complete(ResidentGroup& rg, wf_status st);
  void retire(size_t i, wf_status st);
};

void Server::complete(ResidentGroup& rg, wf_status st) {
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(mu);
  for (size_t i = 0; i < rg.reqs.size(); ++i) {
    auto& r = rg.reqs[i];
    r->status = st != WF_OK ? st : r->info.status;
    r->info.status = r->status;
    r->info.latency_s = std::chrono::duration<double>(now - r->t_submit).count();
  }
  cv_done.notify_all();
}

void Server::run() {
  Ctx& c = *ctx;
  for (;;) {
    // ---- admission (waits only when nothing is resident) ----------------------------------
    std::vector<std::shared_ptr<Request>> admit;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (resident.empty()) cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      if (stop) break;
      while (!queue.empty() && resident_systems + (int)admit.size() < kMaxResident) {
        auto& r = queue.front();
        if (used + r->footprint > budget && !(resident.empty() && admit.empty())) break;
        used += r->footprint;
        admit.push_back(r);
        queue.pop_front();
      }
      resident_systems += (int)admit.size();
    }
    bool progressed = !admit.empty();
    int inflight = 0;
    {
      std::lock_guard<std::mutex> ck(c.mu);
      DeviceGuard dg(c.device);
      // new groups from the admitted requests, by (size, precision): start their preparation
      std::map<std::tuple<int, int, int>, std::vector<std::shared_ptr<Request>>> by;
      for (auto& r : admit) by[{r->args.grid.n, (int)r->args.opts.prec, r->args.opts.deflate}].push_back(r);
      for (auto& kv : by) {
        ResidentGroup rg;
        rg.g.reset(make_group_n(std::get<0>(kv.first), std::get<1>(kv.first)));
        rg.g->tag = "srv" + std::to_string(next_group++) + "_";
        for (auto& r : kv.second) {
          rg.g->sys.push_back(&r->args);
          rg.g->info.push_back(&r->info);
          rg.footprint += r->footprint;
        }
        rg.reqs = kv.second;
        if (free_streams.empty()) free_streams.push_back(next_stream++);
        rg.stream_idx = free_streams.back();
        free_streams.pop_back();
        wf_status st = c.stream(rg.stream_idx, &rg.stream);
        if (st == WF_OK && cudaEventCreateWithFlags(&rg.ev, cudaEventDisableTiming) != cudaSuccess) st = WF_ERR_CUDA;
        if (st == WF_OK) st = rg.g->prepare_begin(c, rg.stream);
        if (st == WF_OK && cudaEventRecord(rg.ev, rg.stream) != cudaSuccess) st = WF_ERR_CUDA;
        rg.state = RG_PREP;
        rg.inflight = true;
        resident.push_back(std::move(rg));
        if (st != WF_OK) retire(resident.size() - 1, st);
      }
      // ---- every group whose device work has finished takes its next step ------------------
      for (size_t i = 0; i < resident.size();) {
        ResidentGroup& rg = resident[i];
        wf_status st = WF_OK;
        if (rg.inflight) {
          const cudaError_t q = cudaEventQuery(rg.ev);
          if (q == cudaErrorNotReady) {
            ++inflight;
            ++i;
            continue;
          }
          rg.inflight = false;
          progressed = true;
          if (q != cudaSuccess) st = WF_ERR_CUDA;
          else if (rg.state == RG_PREP) {
            st = rg.g->prepare_end(c, rg.stream);
            rg.state = RG_RUN;
          } else if (rg.state == RG_RUN) {
            st = rg.g->advance(c);
          } else {  // RG_FIN: the solutions are in the requests' buffers
            retire(i, WF_OK);
            continue;
          }
        }
        if (st == WF_OK && rg.state == RG_RUN) {
          if (rg.g->done()) {
            st = rg.g->finish(c, rg.stream);
            rg.state = RG_FIN;
          } else {
            st = rg.g->enqueue(c, rg.stream);
          }
          if (st == WF_OK && cudaEventRecord(rg.ev, rg.stream) != cudaSuccess) st = WF_ERR_CUDA;
          rg.inflight = true;
          ++inflight;
        }
        if (st != WF_OK) {
          retire(i, st);
          continue;
        }
        ++i;
      }
    }
    // nothing finished on the device since the last pass: let it work a little
    if (!progressed && inflight > 0) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  // shutdown: fail whatever is still queued or resident
  std::lock_guard<std::mutex> lk(mu);
  for (auto& r : queue) r->status = WF_ERR_TIMEOUT;
  for (auto& rg : resident)
    for (auto& r : rg.reqs) r->status = WF_ERR_TIMEOUT;
  cv_done.notify_all();
}

// Complete resident group i with status st (the requests' own status when st is OK), release
// its device memory, stream and event, and drop it.  Scheduler thread, context lock held.
void Server::retire(size_t i, wf_status st) {
  ResidentGroup& rg = resident[i];
  if (rg.inflight && rg.ev) cudaEventSynchronize(rg.ev);  // nothing of it may still run
  complete(rg, st);
  ctx->release_prefix(rg.g->tag);
  if (rg.ev) cudaEventDestroy(rg.ev);
  {
    std::lock_guard<std::mutex> lk(mu);
    used -= rg.footprint;
    resident_systems -= (int)rg.reqs.size();
  }
  free_streams.push_back(rg.stream_idx);
  resident.erase(resident.begin() + i);
}

void serve_shutdown(Ctx& c) {
  Server* s = c.server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  {
    std::lock_guard<std::mutex> ck(c.mu);
    for (auto& rg : s->resident) c.release_prefix(rg.g->tag);
  }
  delete s;
  c.server = nullptr;
}

static Server* server_of(Ctx& c) {
  if (!c.server) {
    Server* s = new Server();
    s->ctx = &c;
    size_t fr = 0, tot = 0;
    {
      DeviceGuard dg(c.device);
      cudaMemGetInfo(&fr, &tot);
    }
    s->budget = c.budget ? c.budget : (size_t)(0.8 * (double)fr);
    c.server = s;
    s->th = std::thread([s] { s->run(); });
  }
  return c.server;
}

}  // namespace wf

using namespace wf;

extern "C" {

wf_status wf_submit(wf_ctx* ctx, const wf_grid* grid, const wf_power* power, const double* w, double nbar,
                    const double* b, const wf_solve_opts* opts, uint64_t* request_id) {
  if (!ctx || !request_id || !grid || !power || !w || !b || !opts) return WF_ERR_ARG;
  if (!supported_size(grid->n)) return WF_ERR_UNSUPPORTED;
  if (!power->k || !power->p || power->n < 2) return WF_ERR_ARG;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  auto r = std::make_shared<Request>();
  const size_t V = (size_t)grid->n * grid->n * grid->n;
  r->V = V;
  r->buf.alloc(3 * V);
  r->w = r->buf.p;
  r->b = r->buf.p + V;
  r->s = r->buf.p + 2 * V;
  std::memcpy(r->w, w, V * sizeof(double));
  std::memcpy(r->b, b, V * sizeof(double));
  r->k.assign(power->k, power->k + power->n);
  r->p.assign(power->p, power->p + power->n);
  wf_power pw{r->k.data(), r->p.data(), power->n};
  wf_status st = prepare_solve(grid, &pw, r->w, nbar, r->b, opts, r->s, r->args);
  if (st != WF_OK) return st;
  r->footprint = Group::footprint(grid->n, (int)opts->prec, 1, r->args.opts.deflate);
  r->t_submit = Clock::now();
  Server* s = server_of(c);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->queue.size() >= kMaxQueued) return WF_ERR_BUSY;
    r->id = s->next_id++;
    s->requests[r->id] = r;
    s->queue.push_back(r);
    *request_id = r->id;
  }
  s->cv_work.notify_one();
  return WF_OK;
}

wf_status wf_poll(wf_ctx* ctx, uint64_t request_id, int timeout_ms, double* s_out, wf_solve_info* info) {
  if (!ctx) return WF_ERR_ARG;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  Server* s = c.server;
  if (!s) return WF_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) return WF_ERR_ARG;
  std::shared_ptr<Request> r = it->second;
  auto ready = [&] { return r->status != WF_PENDING; };
  if (!ready()) {
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  if (!ready()) return WF_PENDING;
  if (s_out) std::memcpy(s_out, r->s, r->V * sizeof(double));
  if (info) *info = r->info;
  const wf_status st = r->status;
  s->requests.erase(it);
  return st;
}

}  // extern "C"
