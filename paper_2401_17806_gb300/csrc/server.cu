// C-ABI of the batched engine (dgsl_cg_solve_batch) and of the request loop
// (dgsl_server_*): host-side admission by memory budget, publication to the
// persistent engine through a mapped inbox, completion collection.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>

#include "kbatch.h"
#include "operator.h"

using namespace dgsl;

namespace {

// Engine resources on one device: mapped inbox and completion records, device
// slot table / state / lists.
struct EngineRes {
  int device = -1;
  BInbox* inbox_h = nullptr;
  BInbox* inbox_d = nullptr;
  BCompletion* done_h = nullptr;
  BCompletion* done_d = nullptr;
  void* area = nullptr;
  EngineParams P{};
  ~EngineRes() {
    if (device < 0) return;
    cudaSetDevice(device);
    if (inbox_h) cudaFreeHost(inbox_h);
    if (done_h) cudaFreeHost(done_h);
    if (area) cudaFree(area);
  }
  void init(int dev) {
    device = dev;
    DGSL_CUDA(cudaSetDevice(dev));
    DGSL_CUDA(cudaHostAlloc(&inbox_h, sizeof(BInbox), cudaHostAllocMapped));
    DGSL_CUDA(cudaHostGetDevicePointer((void**)&inbox_d, inbox_h, 0));
    DGSL_CUDA(cudaHostAlloc(&done_h, sizeof(BCompletion) * kMaxSlots, cudaHostAllocMapped));
    DGSL_CUDA(cudaHostGetDevicePointer((void**)&done_d, done_h, 0));
    std::memset(inbox_h, 0, sizeof(BInbox));
    std::memset(done_h, 0, sizeof(BCompletion) * kMaxSlots);
    DGSL_CUDA(cudaMalloc(&area, engine_state_bytes()));
    engine_layout(area, P);
    P.inbox = inbox_d;
    P.done = done_d;
    P.timeout_ns = 10ull * 1000 * 1000 * 1000;
    P.idle_ns = 0;
  }
  cudaError_t launch(int bf16, int precond, uint64_t idle_ns, cudaStream_t s, int* grid) {
    cudaError_t e = cudaMemsetAsync(P.sh, 0, engine_shared_bytes(), s);
    if (e != cudaSuccess) return e;
    EngineParams q = P;
    q.idle_ns = idle_ns;
    return launch_engine(q, bf16, precond, s, grid);
  }
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

int request_nrhs(const dgsl_request& r) { return r.n_rhs < 1 ? 1 : r.n_rhs; }

// Device workspace of one request (engine_workspace_bytes: FP64 residuals,
// padded FP32 CG vectors, per-chunk partial sums).
size_t request_workspace(const dgsl_operator* op, int nrhs, int precond) {
  return align256(engine_workspace_bytes(op->d.p, op->d.ne, nrhs, precond));
}

int precond_type(const dgsl_engine_opts& o) { return o.precision == DGSL_PREC_BF16_IR ? 2 : 0; }
double request_coefK(const dgsl_request& r) { return r.kind == DGSL_SCHUR ? r.coef * r.coef : r.coef; }
double request_coefM(const dgsl_request& r) { return r.kind == DGSL_SCHUR ? 0.0 : 1.0; }

// Preconditioned operator of a request's system, held until released (builds
// it on stream s if the operator does not keep it).
dgsl_operator::Work::Precond* hold_precond(const dgsl_request& r, const dgsl_engine_opts& o, cudaStream_t s) {
  dgsl_operator* op = const_cast<dgsl_operator*>(r.op);
  std::lock_guard<std::mutex> lock(op->mu);
  return op->acquire_precond(request_coefK(r), request_coefM(r), precond_type(o), s);
}

int check_request(const dgsl_request& r, const dgsl_engine_opts& o, std::string& why) {
  if (!r.op) return why = "request has no operator", DGSL_EINVAL;
  if (r.op->host_only) return why = "operator was built host-only", DGSL_ENODEVICE;
  if (r.op->d.device != o.device) return why = "operator lives on another device", DGSL_EINVAL;
  if (!r.b || !r.x) return why = "request vectors must be non-NULL", DGSL_EINVAL;
  if (r.n_rhs < 0 || r.n_rhs > kMaxRhs) return why = "n_rhs must be 0..8", DGSL_EINVAL;
  if (r.kind != DGSL_SCHUR && r.kind != DGSL_HELMHOLTZ) return why = "bad request kind", DGSL_EINVAL;
  if (!(r.coef >= 0.0) || !std::isfinite(r.coef)) return why = "coef must be finite and >= 0", DGSL_EINVAL;
  if (!r.op->d.K64) return why = "FP64 couplings are needed", DGSL_EINVAL;
  if (o.precision == DGSL_PREC_BF16_IR ? !r.op->d.K16 : !r.op->d.K32)
    return why = "operator lacks the couplings of the engine precision", DGSL_EINVAL;
  return DGSL_OK;
}

int check_engine_opts(const dgsl_engine_opts& o, std::string& why) {
  if (o.precision != DGSL_PREC_F32_IR && o.precision != DGSL_PREC_BF16_IR)
    return why = "engine precision must be DGSL_PREC_F32_IR or DGSL_PREC_BF16_IR", DGSL_EINVAL;
  if (!(o.inner_tol > 0.0) || o.max_iters < 1 || o.max_refine < 1) return why = "bad engine options", DGSL_EINVAL;
  if (o.precond != DGSL_PRECOND_NONE && o.precond != DGSL_PRECOND_BLOCK_JACOBI && o.precond != DGSL_PRECOND_MULTIGRID)
    return why = "precond must be DGSL_PRECOND_NONE, DGSL_PRECOND_BLOCK_JACOBI or DGSL_PRECOND_MULTIGRID",
           DGSL_EINVAL;
  return DGSL_OK;
}

// ---- multigrid requests: concurrent solves, one per worker stream
// A multigrid solve is a sequence of short launches per iteration (the
// V-cycle's levels), not one persistent kernel, so multigrid requests are not
// packed into the engine: each runs the library's solve on a worker's own
// stream, and the solves of different operators overlap on the device.
// Requests on one operator run one at a time (they share its workspace).
constexpr int kMGWorkers = 8;

// Device bytes an operator may grow by at its first multigrid solve of a
// system (the solve workspace, the vertex topology, the smoother blocks, the
// 12 coefficients per row of A Pc, the six fine vectors; the coarse levels are
// small): an upper estimate for admission.
int64_t mg_growth_estimate(const dgsl_operator* op, int precision) {
  const DevOp& d = op->d;
  const int64_t vb = precision == DGSL_PREC_F64 ? 8 : 4, vp = 16 / vb;
  const int64_t work = 24 * d.n + (int64_t)cg_vec_bytes(d, 1) + 64 * 1024;
  const int64_t topo = 24 * (int64_t)d.ne + 64 * 1024;
  const int64_t sys = ((d.nphi + vp - 1) / vp) * d.n * 16 + 12 * d.n * vb + 6 * d.n * vb + 3 * (int64_t)d.ne * vb +
                      (int64_t)d.ne * 40 + 8 * 1024 * 1024;
  return work + topo + sys;
}

// The request's solves (one per right-hand side) with the multigrid
// preconditioner on stream s; the combined info as for engine requests.
void run_mg_request(const dgsl_request& r, const dgsl_engine_opts& o, cudaStream_t s, dgsl_solve_info* info) {
  const int nr = request_nrhs(r);
  dgsl_solve_opts so;
  dgsl_default_solve_opts(&so);
  so.tol = r.tol > 0.0 ? r.tol : 1e-10;
  so.precision = o.precision;
  so.precond = DGSL_PRECOND_MULTIGRID;
  so.inner_tol = o.inner_tol;
  so.max_iters = o.max_iters;
  so.max_refine = o.max_refine;
  std::vector<dgsl_solve_info> each(nr);
  const int st = dgsl_cg_solve(r.op, r.kind, r.coef, r.b, r.x, nr, &so, each.data(), s);
  dgsl_solve_info out{};
  out.status = st;
  for (const auto& e : each) {
    out.iters = std::max(out.iters, e.iters);
    out.refinements = std::max(out.refinements, e.refinements);
    out.cg_launches += e.cg_launches;
    out.relres = std::max(out.relres, e.relres);
    out.cg_kernel_ms += e.cg_kernel_ms;
    out.relres_floor = std::max(out.relres_floor, e.relres_floor);
  }
  *info = out;
}

// held: the request's preconditioned operator (precond), else nullptr.
BSlotDesc fill_desc(const dgsl_request& r, const dgsl_engine_opts& o, char* ws, uint64_t ticket,
                    const dgsl_operator::Work::Precond* held) {
  const DevOp& d = r.op->d;
  BSlotDesc s{};
  s.p = d.p;
  s.ne = d.ne;
  s.ne_pad = d.ne_pad;
  s.mean_zero = r.kind == DGSL_SCHUR;
  s.n = d.n;
  s.nrhs = request_nrhs(r);
  s.K64 = d.K64;
  s.Kin = o.precision == DGSL_PREC_BF16_IR ? (const void*)d.K16 : (const void*)d.K32;
  s.cols = d.cols;
  s.area = d.area;
  s.Mref = d.Mref;
  s.coefK = request_coefK(r);
  s.coefM = request_coefM(r);
  if (held) {
    s.precond = 1;
    s.Kin = held->op.ap;
    s.Pin = static_cast<const float*>(held->op.pinv);
  }
  s.b = r.b;
  s.x = r.x;
  s.tol = r.tol > 0.0 ? r.tol : 1e-10;
  s.inner_tol = o.inner_tol;
  s.max_iters = o.max_iters;
  s.max_refine = o.max_refine;
  s.ticket = (long long)ticket;
  engine_fill_workspace(s, ws);
  return s;
}

void info_from(const BCompletion& c, dgsl_solve_info* info) {
  info->status = c.status;
  info->iters = c.iters;
  info->refinements = c.refinements;
  info->cg_launches = 1;
  info->relres = c.relres;
  info->cg_kernel_ms = 0.0;
  info->grid = 0;
  info->pad = 0;
  info->relres_floor = 0.0;
}

std::mutex g_batch_mu;
std::map<int, std::unique_ptr<EngineRes>> g_batch_engines;

}  // namespace

extern "C" void dgsl_default_engine_opts(dgsl_engine_opts* o) {
  if (!o) return;
  o->precision = DGSL_PREC_F32_IR;
  o->max_iters = 200000;
  o->inner_tol = 1e-3;
  o->max_refine = 30;
  o->device = 0;
  o->hbm_budget_bytes = 150000000000LL;
  o->idle_us = 500;
  o->precond = DGSL_PRECOND_NONE;
  o->pad = 0;
}

extern "C" int dgsl_cg_solve_batch(const dgsl_request* reqs, int n, const dgsl_engine_opts* opts,
                                   dgsl_solve_info* infos, void* stream) {
  NvtxRange nvtx("dgsl_cg_solve_batch");
  dgsl_engine_opts o;
  dgsl_default_engine_opts(&o);
  if (opts) o = *opts;
  try {
    if (!reqs || n < 1 || n > kMaxSlots) throw Error(DGSL_EINVAL, "need 1..4096 requests");
    std::string why;
    if (int e = check_engine_opts(o, why)) throw Error(e, why);
    for (int i = 0; i < n; ++i)
      if (int e = check_request(reqs[i], o, why)) throw Error(e, "request " + std::to_string(i) + ": " + why);
    if (o.precond == DGSL_PRECOND_MULTIGRID) {
      // requests of one operator run in order on one worker; operators spread
      // over kMGWorkers streams
      DGSL_CUDA(cudaSetDevice(o.device));
      cudaStream_t s0 = (cudaStream_t)stream;
      DGSL_CUDA(cudaStreamSynchronize(s0));  // the inputs are ready before the worker streams read them
      std::vector<std::vector<int>> lanes(kMGWorkers);
      std::unordered_map<const dgsl_operator*, int> lane_of;
      for (int i = 0; i < n; ++i) {
        auto it = lane_of.find(reqs[i].op);
        const int l = it != lane_of.end() ? it->second : (int)(lane_of.size() % kMGWorkers);
        lane_of.emplace(reqs[i].op, l);
        lanes[l].push_back(i);
      }
      std::vector<dgsl_solve_info> out(n);
      std::vector<std::thread> th;
      std::atomic<int> failed{0};
      for (int l = 0; l < kMGWorkers; ++l) {
        if (lanes[l].empty()) continue;
        th.emplace_back([&, l] {
          cudaSetDevice(o.device);
          cudaStream_t ws = nullptr;
          if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            failed = 1;
            return;
          }
          for (int i : lanes[l]) run_mg_request(reqs[i], o, ws, &out[i]);
          cudaStreamSynchronize(ws);
          cudaStreamDestroy(ws);
        });
      }
      for (auto& t : th) t.join();
      if (failed) throw Error(DGSL_ECUDA, "could not create a worker stream");
      int worst = DGSL_OK;
      for (int i = 0; i < n; ++i) {
        if (infos) infos[i] = out[i];
        if (out[i].status != DGSL_OK && worst == DGSL_OK) worst = out[i].status;
      }
      if (worst != DGSL_OK) dgsl_set_last_error("at least one request did not converge (see infos)");
      return worst;
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    DGSL_CUDA(cudaSetDevice(o.device));
    auto& R = g_batch_engines[o.device];
    if (!R) {
      R = std::make_unique<EngineRes>();
      R->init(o.device);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // preconditioned operators, held for the whole call
    std::vector<dgsl_operator::Work::Precond*> held(n, nullptr);
    struct Release {
      std::vector<dgsl_operator::Work::Precond*>& h;
      ~Release() {
        for (auto* c : h) dgsl_operator::release_precond(c);
      }
    } release{held};
    if (o.precond)
      for (int i = 0; i < n; ++i) held[i] = hold_precond(reqs[i], o, s);
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
      off[i] = total;
      total += request_workspace(reqs[i].op, request_nrhs(reqs[i]), o.precond);
    }
    char* ws = nullptr;
    if (cudaMalloc(&ws, total) != cudaSuccess) throw Error(DGSL_ENOMEM, "batch workspace allocation failed");
    std::unique_ptr<char, void (*)(char*)> guard(ws, [](char* q) { cudaFree(q); });
    for (int i = 0; i < n; ++i) R->inbox_h->slots[i] = fill_desc(reqs[i], o, ws + off[i], (uint64_t)i, held[i]);
    std::memset(R->done_h, 0, sizeof(BCompletion) * kMaxSlots);
    R->inbox_h->stop = 1;
    std::atomic_thread_fence(std::memory_order_release);
    R->inbox_h->count = n;
    int grid = 0;
    DGSL_CUDA(R->launch(o.precision == DGSL_PREC_BF16_IR, o.precond, 0, s, &grid));
    DGSL_CUDA(cudaStreamSynchronize(s));
    std::vector<char> sh(engine_shared_bytes());
    DGSL_CUDA(cudaMemcpy(sh.data(), R->P.sh, sh.size(), cudaMemcpyDeviceToHost));
    const int engine_status = engine_shared_status(sh.data());
    int worst = DGSL_OK;
    for (int i = 0; i < n; ++i) {
      BCompletion c = R->done_h[i];
      dgsl_solve_info tmp;
      if (!c.done) {
        std::memset(&tmp, 0, sizeof(tmp));
        tmp.status = engine_status ? DGSL_ETIMEOUT : DGSL_ENOTCONV;
      } else {
        info_from(c, &tmp);
      }
      tmp.grid = grid;
      if (infos) infos[i] = tmp;
      if (tmp.status != DGSL_OK && worst == DGSL_OK) worst = tmp.status;
    }
    R->inbox_h->count = 0;
    R->inbox_h->stop = 0;
    if (worst != DGSL_OK) dgsl_set_last_error("at least one request did not converge (see infos)");
    return worst;
  } catch (const Error& e) {
    dgsl_set_last_error(e.what());
    return e.code;
  }
}

// ------------------------------------------------------------ request loop

namespace {

// First-fit allocator over the server's device workspace arena (host-side
// bookkeeping only; the arena is one allocation made at create time).
struct Arena {
  char* base = nullptr;
  size_t bytes = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  void init(char* b, size_t n) {
    base = b;
    bytes = n;
    free_.clear();
    free_[0] = n;
  }
  char* alloc(size_t n) {
    n = align256(n);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= n) {
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > n) free_[off + n] = sz - n;
        return base + off;
      }
    return nullptr;
  }
  void release(char* p, size_t n) {
    n = align256(n);
    size_t off = (size_t)(p - base);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }
};

enum { RQ_QUEUED = 0, RQ_ADMITTED = 1, RQ_DONE = 2 };

struct Request {
  dgsl_request r{};
  uint64_t ticket = 0;
  int state = RQ_QUEUED;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  dgsl_operator::Work::Precond* held = nullptr;  // preconditioned operator while admitted
  dgsl_solve_info info{};
};

// Operators of the requests in flight: how many, and the device bytes charged
// to the budget for each (its size when first admitted, plus any growth from
// preconditioned operators built for later requests).
struct OpRef {
  int count = 0;
  int64_t charged = 0;
};

}  // namespace

struct dgsl_server {
  dgsl_engine_opts o{};
  EngineRes R;
  cudaStream_t stream = nullptr;
  cudaStream_t build_stream = nullptr;  // preconditioned operators are built here
  cudaEvent_t exited = nullptr;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> queue;
  std::unordered_map<const dgsl_operator*, OpRef> op_refs;  // operators of requests in flight
  int64_t bytes_in_use = 0;
  bool running = false;
  int published = 0;                      // slots published to the current launch
  std::vector<uint64_t> slot_ticket;      // [kMaxSlots]
  std::vector<char> collected;            // [kMaxSlots]
  std::vector<char> slot_late;            // [kMaxSlots] published while the launch was already running
  int64_t submitted = 0, completed = 0, launches = 0;
  int64_t admitted_running = 0;           // late slots the running engine admitted and finished
  // multigrid mode: worker threads, each with its own stream, admitting
  // requests while the other workers' solves run
  bool mg_mode = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> wstreams;
  std::set<const dgsl_operator*> busy;    // operators with a solve running
  int active = 0;                         // solves running

  void worker(int w) {
    cudaSetDevice(o.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      // the first queued request whose operator is free and which fits the budget
      auto pick = queue.end();
      int64_t need = 0;
      for (auto it = queue.begin(); it != queue.end(); ++it) {
        Request& q = reqs[*it];
        if (busy.count(q.r.op)) continue;
        need = op_cost(q.r.op) + mg_growth_estimate(q.r.op, o.precision);
        if (bytes_in_use + need <= o.hbm_budget_bytes || active == 0) {
          pick = it;
          break;
        }
        break;  // in order: a request that does not fit waits for memory, later ones wait behind it
      }
      if (pick == queue.end()) {
        if (stopping && queue.empty()) return;
        cv.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
      const uint64_t t = *pick;
      queue.erase(pick);
      Request& q = reqs[t];
      q.state = RQ_ADMITTED;
      busy.insert(q.r.op);
      OpRef& ref = op_refs[q.r.op];
      ++ref.count;
      ref.charged += need;
      bytes_in_use += need;
      const bool late = active > 0;  // joins solves already on the device
      ++active;
      ++launches;
      const dgsl_request r = q.r;
      const int64_t before = r.op->device_bytes;
      lk.unlock();
      dgsl_solve_info info{};
      run_mg_request(r, o, wstreams[w], &info);
      cudaStreamSynchronize(wstreams[w]);
      lk.lock();
      // the estimate becomes the operator's actual growth
      OpRef& rf = op_refs[r.op];
      const int64_t actual = r.op->device_bytes - before;
      bytes_in_use += actual - mg_growth_estimate(r.op, o.precision);
      rf.charged += actual - mg_growth_estimate(r.op, o.precision);
      Request& qd = reqs[t];
      qd.info = info;
      qd.state = RQ_DONE;
      ++completed;
      if (late) ++admitted_running;
      if (--rf.count == 0) {
        bytes_in_use -= rf.charged;
        op_refs.erase(r.op);
      }
      busy.erase(r.op);
      --active;
      cv.notify_all();
    }
  }

  // Device bytes of op not yet charged to the budget.
  int64_t op_cost(const dgsl_operator* op) const {
    auto it = op_refs.find(op);
    return op->device_bytes - (it == op_refs.end() ? 0 : it->second.charged);
  }

  // Gives back a request's workspace, its hold on the preconditioned operator
  // and its reference to the operator.
  void unadmit(Request& q) {
    arena.release(q.ws, q.ws_bytes);
    bytes_in_use -= (int64_t)q.ws_bytes;
    dgsl_operator::release_precond(q.held);
    q.held = nullptr;
    q.ws = nullptr;
    OpRef& ref = op_refs[q.r.op];
    if (--ref.count == 0) {
      bytes_in_use -= ref.charged;
      op_refs.erase(q.r.op);
    }
  }

  void finish(Request& q) {
    unadmit(q);
    q.state = RQ_DONE;
    ++completed;
  }

  // One scheduling round (called with mu held).
  void round() {
    NvtxRange nvtx("dgsl server round");
    // 1. engine exit: requeue slots it never admitted, reset the inbox
    if (running && cudaEventQuery(exited) == cudaSuccess) {
      running = false;
      std::vector<char> sh(engine_shared_bytes());
      cudaMemcpy(sh.data(), R.P.sh, sh.size(), cudaMemcpyDeviceToHost);
      const int admitted = engine_shared_admitted(sh.data());
      collect();
      for (int i = published - 1; i >= admitted; --i) {
        Request& q = reqs[slot_ticket[i]];
        unadmit(q);
        q.state = RQ_QUEUED;
        queue.push_front(q.ticket);
      }
      published = 0;
      std::memset(R.done_h, 0, sizeof(BCompletion) * kMaxSlots);
      std::fill(collected.begin(), collected.end(), 0);
      R.inbox_h->stop = 0;
      std::atomic_thread_fence(std::memory_order_release);
      *((volatile int*)&R.inbox_h->count) = 0;
    }
    collect();
    // 2. admission under the budget
    int added = 0;
    while (!queue.empty() && published < kMaxSlots) {
      Request& q = reqs[queue.front()];
      if (o.precond && !q.held) {
        // the operator grows by the preconditioned system the first time
        try {
          q.held = hold_precond(q.r, o, build_stream);
        } catch (const Error& e) {
          q.info = dgsl_solve_info{};
          q.info.status = e.code;
          q.state = RQ_DONE;
          ++completed;
          queue.pop_front();
          continue;
        }
      }
      const int64_t opc = op_cost(q.r.op);
      const int64_t need = (int64_t)q.ws_bytes + opc;
      if (bytes_in_use + need > o.hbm_budget_bytes) break;  // (keeps its hold until admitted)
      char* ws = arena.alloc(q.ws_bytes);
      if (!ws) break;
      q.ws = ws;
      bytes_in_use += need;
      OpRef& ref = op_refs[q.r.op];
      ++ref.count;
      ref.charged += opc;
      q.state = RQ_ADMITTED;
      R.inbox_h->slots[published] = fill_desc(q.r, o, ws, q.ticket, q.held);
      slot_ticket[published] = q.ticket;
      slot_late[published] = running ? 1 : 0;
      ++published;
      ++added;
      queue.pop_front();
    }
    if (added) {
      std::atomic_thread_fence(std::memory_order_release);
      *((volatile int*)&R.inbox_h->count) = published;
    }
    if (published >= kMaxSlots) R.inbox_h->stop = 1;  // drain this launch, then start a new one
    // 3. launch when there is published work and no engine
    if (!running && published > 0) {
      int grid = 0;
      if (R.launch(o.precision == DGSL_PREC_BF16_IR, o.precond, (uint64_t)o.idle_us * 1000ull, stream, &grid) ==
              cudaSuccess &&
          cudaEventRecord(exited, stream) == cudaSuccess) {
        running = true;
        ++launches;
      }
    }
  }

  void collect() {
    for (int i = 0; i < published; ++i) {
      if (collected[i]) continue;
      if (!*((volatile int*)&R.done_h[i].done)) continue;
      std::atomic_thread_fence(std::memory_order_acquire);
      Request& q = reqs[slot_ticket[i]];
      info_from(R.done_h[i], &q.info);
      collected[i] = 1;
      if (slot_late[i]) ++admitted_running;  // a completion means the engine admitted the slot
      finish(q);
    }
  }

  void loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      round();
      if (stopping && queue.empty() && !running) break;
      cv.wait_for(lk, std::chrono::microseconds(running ? 20 : 200));
    }
  }
};

extern "C" int dgsl_server_create(const dgsl_engine_opts* opts, dgsl_server** out) {
  if (!out) return dgsl_set_last_error("out must be non-NULL"), DGSL_EINVAL;
  *out = nullptr;
  try {
    auto s = std::make_unique<dgsl_server>();
    dgsl_default_engine_opts(&s->o);
    if (opts) s->o = *opts;
    if (s->o.hbm_budget_bytes <= 0) s->o.hbm_budget_bytes = 150000000000LL;
    std::string why;
    if (int e = check_engine_opts(s->o, why)) throw Error(e, why);
    if (s->o.idle_us < 0 || s->o.idle_us > 1000000) throw Error(DGSL_EINVAL, "idle_us must be in [0, 1e6]");
    if (s->o.precond == DGSL_PRECOND_MULTIGRID) {
      DGSL_CUDA(cudaSetDevice(s->o.device));
      s->mg_mode = true;
      s->wstreams.resize(kMGWorkers);
      for (auto& w : s->wstreams) DGSL_CUDA(cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking));
      dgsl_server* raw = s.get();
      for (int w = 0; w < kMGWorkers; ++w) s->workers.emplace_back([raw, w] { raw->worker(w); });
      *out = s.release();
      return DGSL_OK;
    }
    s->R.init(s->o.device);
    DGSL_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    DGSL_CUDA(cudaStreamCreateWithFlags(&s->build_stream, cudaStreamNonBlocking));
    DGSL_CUDA(cudaEventCreateWithFlags(&s->exited, cudaEventDisableTiming));
    // workspace arena: the budget minus nothing (operators are owned by the
    // caller), capped by the memory free on the device
    size_t free_b = 0, total_b = 0;
    DGSL_CUDA(cudaMemGetInfo(&free_b, &total_b));
    size_t want = std::min((size_t)s->o.hbm_budget_bytes, free_b / 10 * 9);
    char* base = nullptr;
    if (cudaMalloc(&base, want) != cudaSuccess) throw Error(DGSL_ENOMEM, "server workspace arena allocation failed");
    s->arena.init(base, want);
    s->slot_ticket.assign(kMaxSlots, 0);
    s->collected.assign(kMaxSlots, 0);
    s->slot_late.assign(kMaxSlots, 0);
    dgsl_server* raw = s.get();
    s->th = std::thread([raw] { raw->loop(); });
    *out = s.release();
    return DGSL_OK;
  } catch (const Error& e) {
    dgsl_set_last_error(e.what());
    return e.code;
  }
}

extern "C" int dgsl_submit(dgsl_server* srv, const dgsl_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return dgsl_set_last_error("NULL argument"), DGSL_EINVAL;
  std::string why;
  if (int e = check_request(*req, srv->o, why)) return dgsl_set_last_error(why), e;
  Request q;
  q.r = *req;
  if (srv->mg_mode) {
    if (req->op->device_bytes + mg_growth_estimate(req->op, srv->o.precision) > srv->o.hbm_budget_bytes)
      return dgsl_set_last_error("request can never fit the memory budget"), DGSL_EBUDGET;
    std::lock_guard<std::mutex> lk(srv->mu);
    q.ticket = srv->next_ticket++;
    *ticket = q.ticket;
    srv->queue.push_back(q.ticket);
    srv->reqs.emplace(q.ticket, q);
    ++srv->submitted;
    srv->cv.notify_all();
    return DGSL_OK;
  }
  q.ws_bytes = request_workspace(req->op, request_nrhs(*req), srv->o.precond);
  // with the preconditioner the operator may grow by A P, P and an FP64 P
  const int64_t pre_bytes =
      srv->o.precond ? (int64_t)(precond_ap_bytes(req->op->d, precond_type(srv->o)) +
                                 precond_pinv_bytes(req->op->d, precond_type(srv->o)) + precond_pinv_bytes(req->op->d, 1))
                     : 0;
  if ((int64_t)q.ws_bytes + req->op->device_bytes + pre_bytes > srv->o.hbm_budget_bytes ||
      q.ws_bytes > srv->arena.bytes)
    return dgsl_set_last_error("request can never fit the memory budget"), DGSL_EBUDGET;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    q.ticket = srv->next_ticket++;
    *ticket = q.ticket;
    srv->queue.push_back(q.ticket);
    srv->reqs.emplace(q.ticket, q);
    ++srv->submitted;
  }
  srv->cv.notify_one();
  return DGSL_OK;
}

extern "C" int dgsl_poll(dgsl_server* srv, uint64_t ticket, dgsl_solve_info* info) {
  if (!srv) return dgsl_set_last_error("NULL server"), DGSL_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return dgsl_set_last_error("unknown ticket"), DGSL_EINVAL;
  if (it->second.state != RQ_DONE) return DGSL_EPENDING;
  if (info) *info = it->second.info;
  srv->reqs.erase(it);
  return DGSL_OK;
}

extern "C" int dgsl_poll_many(dgsl_server* srv, const uint64_t* tickets, int n, dgsl_solve_info* infos,
                              int32_t* done) {
  if (!srv || (!tickets && n > 0) || !done || n < 0) return dgsl_set_last_error("bad arguments"), -DGSL_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  int finished = 0;
  for (int i = 0; i < n; ++i) {
    auto it = srv->reqs.find(tickets[i]);
    if (it == srv->reqs.end()) {
      done[i] = -1;
      continue;
    }
    if (it->second.state != RQ_DONE) {
      done[i] = 0;
      continue;
    }
    if (infos) infos[i] = it->second.info;
    done[i] = 1;
    ++finished;
    srv->reqs.erase(it);
  }
  return finished;
}

extern "C" int dgsl_cancel(dgsl_server* srv, uint64_t ticket) {
  if (!srv) return dgsl_set_last_error("NULL server"), DGSL_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return dgsl_set_last_error("unknown ticket"), DGSL_EINVAL;
  if (it->second.state != RQ_QUEUED) return DGSL_EPENDING;
  dgsl_operator::release_precond(it->second.held);  // (a queued request may hold one)
  for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
    if (*q == ticket) {
      srv->queue.erase(q);
      break;
    }
  srv->reqs.erase(it);
  return DGSL_OK;
}

extern "C" int dgsl_server_get_stats(dgsl_server* srv, dgsl_server_stats* out) {
  if (!srv || !out) return dgsl_set_last_error("NULL argument"), DGSL_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->queued = (int64_t)srv->queue.size();
  out->in_flight = srv->submitted - srv->completed - (int64_t)srv->queue.size();
  out->engine_launches = srv->launches;
  out->bytes_in_use = srv->bytes_in_use;
  out->admitted_running = srv->admitted_running;
  return DGSL_OK;
}

extern "C" void dgsl_server_destroy(dgsl_server* srv) {
  if (!srv) return;
  if (srv->mg_mode) {
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->stopping = true;
    }
    srv->cv.notify_all();
    for (auto& t : srv->workers) t.join();
    cudaSetDevice(srv->o.device);
    for (auto w : srv->wstreams) cudaStreamDestroy(w);
    delete srv;
    return;
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
    srv->R.inbox_h->stop = 1;
  }
  srv->cv.notify_one();
  if (srv->th.joinable()) srv->th.join();
  cudaSetDevice(srv->o.device);
  cudaStreamSynchronize(srv->stream);
  cudaFree(srv->arena.base);
  for (auto& kv : srv->reqs) dgsl_operator::release_precond(kv.second.held);
  cudaEventDestroy(srv->exited);
  cudaStreamDestroy(srv->stream);
  cudaStreamDestroy(srv->build_stream);
  delete srv;
}
