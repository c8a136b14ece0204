// mf_server.cu -- continuous-batching solve server.
//
// Requests (a mesh, degree, operator kind, geometry, right-hand side and tolerance) are
// queued by mf_batch_submit and admitted in arrival order whenever a slot and enough of the
// caller's device arena are free; a request that does not fit yet does not block smaller
// ones behind it.  Each admitted request keeps its geometry, vectors and CG state resident
// in its own arena block and runs the solver engine (FP64 CG, or FP32 CG inside FP64
// defect correction).  Its set-up, outer defect-correction steps and finish run on its
// slot's stream.  Its CG iterations run in a continuous batch: the requests in the inner-CG
// phase are grouped by class (degree, path, kind, vector type, launch variant), and each
// class runs chunks of batched iterations -- one launch per kernel for all its members --
// on the class's stream; requests join and leave between chunks.  A scheduler thread
// (native) polls one event per slot and per class, advances requests when their scalars
// have landed, admits new requests as slots and memory free up, and retires finished ones.
//
// Results (status, iterations, residual, L2 error for manufactured right-hand sides, and the
// submit / admit / finish times) are kept until mf_batch_poll has returned them.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "mf_internal.h"
#include "mf_solver.h"

namespace mf {
namespace {

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

// First-fit allocator over the caller's device arena (offsets, 256-byte granules,
// neighbouring free blocks coalesced on release).
class Arena {
 public:
  void init(char* base, size_t bytes) {
    base_ = base;
    size_ = bytes & ~size_t(255);
    free_.clear();
    if (size_) free_[0] = size_;
    used_ = peak_ = 0;
  }
  char* alloc(size_t bytes) {
    bytes = a256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_ += bytes;
      if (used_ > peak_) peak_ = used_;
      return base_ + off;
    }
    return nullptr;
  }
  void release(char* p, size_t bytes) {
    bytes = a256(bytes);
    size_t off = (size_t)(p - base_);
    used_ -= bytes;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + bytes == nx->first) {
      bytes += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        pv->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  char* base_ = nullptr;
  size_t size_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

__global__ void random_unique_kernel(double* u, long long n, unsigned long long seed) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
    // splitmix64 counter stream: draw m of seed s (same definition as the Python inputs module)
    unsigned long long z = seed + (unsigned long long)(m + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    u[m] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
  }
}

enum Stage { ST_QUEUED = 0, ST_SOLVING = 1, ST_FINISHING = 2, ST_DONE = 3 };

// Requests whose apply launches at most this many CTAs join continuous batches (about two
// waves of two CTAs per SM on 152 SMs).
constexpr long long BATCH_MAX_CTAS = 1024;

struct Job {
  uint64_t ticket = 0;
  mf_request req{};
  double t_submit = 0, t_admit = -1, t_done = -1;
  int stage = ST_QUEUED;
  int slot = -1;
  mf_status status = MF_ERR_BUSY;
  mf_mesh* mesh = nullptr;
  mf_operator* op = nullptr;
  mf_info info{};
  size_t bytes = 0;
  char* mem = nullptr;
  void *opws = nullptr, *b = nullptr, *x = nullptr, *cgws = nullptr, *mws = nullptr, *xu = nullptr;
  size_t opws_b = 0, cgws_b = 0, mws_b = 0;
  SolverEngine eng;
  double l2 = -1.0;
  bool cancel = false;
  long long steps = 0, max_steps = 0; // engine advances (bounded: see job_start)
  bool batch_ready = false;           // in the inner CG with scalars landed: joins the next chunk
  bool in_batch = false;              // a chunk of its class is in flight
};

// A class of requests whose CG iterations share batched launches.
struct BatchClass {
  int n = 0, path = 0, kind = 0, elem = 0, variant = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  int cap = 0;              // members the buffers hold
  char* dev = nullptr;      // arena: descriptors, then the gathered states
  size_t dev_bytes = 0;
  char* host = nullptr;     // pinned: descriptor staging, then the states read back
  size_t host_bytes = 0, states_off = 0;
  std::vector<Job*> members;      // of the chunk in flight
  std::vector<uint64_t> planned;  // tickets whose descriptors are on the device
  BatchPlan plan;
  bool running = false;
  cudaGraphExec_t exec = nullptr; // one iteration of the planned composition
  bool exec_current = false;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  Job* job = nullptr;
};

} // namespace
} // namespace mf

struct mf_server {
  mf_server_config cfg{};
  int device = 0;
  mf::Arena arena;
  std::vector<mf::Slot> slots;
  mf::HostMirror* mirrors = nullptr; // pinned, one per slot
  double* l2_host = nullptr;         // pinned, one per slot
  std::mutex mu;
  std::condition_variable cv;
  std::deque<mf::Job*> pending;
  std::map<uint64_t, mf::Job*> jobs;
  uint64_t next_ticket = 1;
  std::vector<mf::BatchClass*> classes;
  std::thread th;
  std::atomic<bool> stop{false};
  std::chrono::steady_clock::time_point t0;
  long long admitted = 0, completed = 0;
  mf_status thread_error = MF_OK;
};

namespace mf {
namespace {

double now_s(const mf_server* sv) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - sv->t0).count();
}

// Host objects and footprint of a request (no device work).
mf_status job_prepare(mf_server* sv, Job* j) {
  const mf_request& r = j->req;
  mf_status st = mf_mesh_create(r.nx, r.ny, r.nz, r.geometry, nullptr, r.curve_amp, &j->mesh);
  if (st) return st;
  st = mf_operator_create(j->mesh, r.degree, r.kind, r.mass_coeff, r.mixed ? MF_MIXED : MF_FP64, MF_BC_DIRICHLET0, &j->op);
  if (st) return st;
  mf_operator_info(j->op, &j->info);
  j->opws_b = a256(j->info.workspace_bytes);
  j->cgws_b = a256(mf_cg_workspace_bytes(j->op, r.mixed ? 1 : 0));
  j->mws_b = a256(mf_manufactured_workspace_bytes(j->op));
  const size_t vec = a256((size_t)j->info.n_native * 8);
  const size_t uvec = a256((size_t)j->info.n_unique * 8);
  j->bytes = j->opws_b + j->cgws_b + j->mws_b + 2 * vec + uvec;
  if (j->bytes > sv->arena.size())
    return set_error(MF_ERR_OOM, "request needs %zu device bytes, arena holds %zu", j->bytes, sv->arena.size());
  return MF_OK;
}

void job_free_host(Job* j) {
  if (j->op) mf_operator_destroy(j->op);
  if (j->mesh) mf_mesh_destroy(j->mesh);
  j->op = nullptr;
  j->mesh = nullptr;
}

// Device set-up on the slot stream: geometry, right-hand side, solver start.
mf_status job_start(mf_server* sv, Job* j, Slot& sl, HostMirror* hm) {
  char* p = j->mem;
  j->opws = p; p += j->opws_b;
  j->cgws = p; p += j->cgws_b;
  j->mws = p; p += j->mws_b;
  j->b = p; p += a256((size_t)j->info.n_native * 8);
  j->x = p; p += a256((size_t)j->info.n_native * 8);
  j->xu = p;
  cudaStream_t s = sl.s;
  mf_status st = mf_operator_setup(j->op, j->opws, j->opws_b, s);
  if (st) return st;
  if (j->req.rhs == MF_RHS_RANDOM) {
    random_unique_kernel<<<1024, 256, 0, s>>>((double*)j->xu, j->info.n_unique, (unsigned long long)j->req.seed);
    if ((st = cuda_check(cudaGetLastError(), "random rhs"))) return st;
    if ((st = mf_scatter_unique(j->op, j->xu, j->b, s))) return st;
  } else {
    if ((st = mf_rhs_manufactured(j->op, j->req.freq, j->b, j->mws, j->mws_b, s))) return st;
  }
  if (sv->cfg.autotune) {
    // times both launch variants on b (x is overwritten; the solve starts from zero)
    if ((st = mf_operator_autotune(j->op, j->b, j->x, 2, s))) return st;
  }
  engine_init(&j->eng, j->op, j->req.mixed ? 1 : 0, j->b, j->x, j->req.rtol, j->req.maxit, j->cgws, s, hm);
  // chunks of 10 iterations by default: a member that converges mid-chunk idles less (the
  // 100-request burst: p50 5.7 -> 4.1 s against 20)
  j->eng.chunk = sv->cfg.chunk_iterations > 0 ? sv->cfg.chunk_iterations : 10;
  if (sv->cfg.inner_rtol > 0) j->eng.inner_rtol = sv->cfg.inner_rtol;
  j->eng.reliable = sv->cfg.mixed_restart == 0;
  // Inner iterations come from the class batches for requests whose apply is a few waves of
  // CTAs at most: those are launch- and latency-bound alone, and batched with others they
  // share launches.  A larger request fills the GPU by itself and runs its own graph chunks
  // (batched with small ones it would hold them to its own chunk time).
  // (the default launch variant puts 8 to 32 cells of a 32-cell tile in one CTA: at most 4
  // CTAs per tile below degree 8)
  const long long ctas = j->op->g.ntiles * 4;
  j->eng.external = sv->cfg.batching >= 0 && ctas <= BATCH_MAX_CTAS;
  if ((st = engine_start(&j->eng))) return st;
  // every advance finishes or moves the iteration count forward by a chunk
  j->max_steps = 2LL * ((long long)j->req.maxit / j->eng.chunk + 2) * (j->eng.max_outer + 2) + 16;
  j->stage = ST_SOLVING;
  return cuda_check(cudaEventRecord(sl.ev, s), "event record");
}

// Engine finished: L2 error (manufactured) and solution copy-out, enqueued on the stream.
mf_status job_finish_enqueue(mf_server* sv, Job* j, Slot& sl, int slot) {
  cudaStream_t s = sl.s;
  mf_status st;
  if (j->req.rhs == MF_RHS_MANUFACTURED && j->eng.status == MF_OK) {
    double* dev = reinterpret_cast<double*>(j->xu); // n_unique >= 1 doubles of scratch
    if ((st = mf_error_manufactured(j->op, j->req.freq, j->x, dev, j->mws, j->mws_b, s))) return st;
    if ((st = cuda_check(cudaMemcpyAsync(&sv->l2_host[slot], dev, sizeof(double), cudaMemcpyDeviceToHost, s), "l2 D2H")))
      return st;
  } else {
    sv->l2_host[slot] = -1.0;
  }
  j->stage = ST_FINISHING;
  return cuda_check(cudaEventRecord(sl.ev, s), "event record");
}

void job_retire(mf_server* sv, Job* j, Slot& sl, int slot) {
  cudaStream_t s = sl.s;
  if (j->req.x_out_host && j->eng.status == MF_OK) {
    if (mf_gather_unique(j->op, j->x, j->xu, s) == MF_OK)
      cudaMemcpyAsync(j->req.x_out_host, j->xu, sizeof(double) * (size_t)j->info.n_unique, cudaMemcpyDeviceToHost, s);
  }
  cudaStreamSynchronize(s);
  engine_release(&j->eng);
  const double l2 = sv->l2_host[slot];
  std::lock_guard<std::mutex> lk(sv->mu);
  j->l2 = l2 >= 0 ? std::sqrt(l2) : -1.0;
  j->status = j->cancel ? MF_ERR_CANCELLED : j->eng.status;
  j->t_done = now_s(sv);
  j->stage = ST_DONE;
  sv->arena.release(j->mem, j->bytes);
  j->mem = nullptr;
  job_free_host(j);
  sl.job = nullptr;
  sv->completed += 1;
  sv->cv.notify_all();
}

void job_fail(mf_server* sv, Job* j, Slot* sl, mf_status st) {
  if (sl) {
    cudaStreamSynchronize(sl->s);
    engine_release(&j->eng);
    sl->job = nullptr;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (j->mem) sv->arena.release(j->mem, j->bytes);
  j->mem = nullptr;
  job_free_host(j);
  j->status = st;
  j->t_done = now_s(sv);
  j->stage = ST_DONE;
  sv->completed += 1;
  sv->cv.notify_all();
}

int class_view(const Job* j) {
  return j->eng.vt == ELEM_DD ? VK_DDS : (j->eng.vt == 4 ? VK_F32 : fp64_view(j->op));
}

// The batch class of a request in its inner CG (created on first use).  nullptr when its
// buffers do not fit: the request then runs its own chunks.  (Up to four concurrent chunks
// per class -- a request ready while its class's chunk is in flight starting another -- were
// measured: no gain on the 100- and 400-request streams.)
BatchClass* class_of(mf_server* sv, const Job* j) {
  const int vk = class_view(j);
  const int variant = j->op->variant[vk == VK_DDS ? VK_DD : vk];
  for (BatchClass* c : sv->classes)
    if (c->n == j->op->n && c->path == j->op->path && c->kind == j->op->kind && c->elem == j->eng.vt &&
        c->variant == variant)
      return c;
  BatchClass* c = new (std::nothrow) BatchClass;
  if (!c) return nullptr;
  c->n = j->op->n;
  c->path = j->op->path;
  c->kind = j->op->kind;
  c->elem = j->eng.vt;
  c->variant = variant;
  c->cap = (int)sv->slots.size();
  const size_t desc = batch_plan_bytes(c->cap, vk);
  c->states_off = desc;
  c->dev_bytes = desc + a256(sizeof(CgState) * (size_t)c->cap);
  c->host_bytes = c->dev_bytes;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    c->dev = sv->arena.alloc(c->dev_bytes);
  }
  bool ok = c->dev != nullptr && cudaMallocHost(&c->host, c->host_bytes) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->s) cudaStreamDestroy(c->s);
    if (c->host) cudaFreeHost(c->host);
    if (c->dev) {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->arena.release(c->dev, c->dev_bytes);
    }
    delete c;
    return nullptr;
  }
  sv->classes.push_back(c);
  return c;
}

void class_destroy(mf_server* sv, BatchClass* c) {
  if (c->s) cudaStreamSynchronize(c->s);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->ev) cudaEventDestroy(c->ev);
  if (c->s) cudaStreamDestroy(c->s);
  if (c->host) cudaFreeHost(c->host);
  (void)sv; // the arena block goes with the arena
  delete c;
}

// After the engine advanced: finish, wait for the next batch, or continue on the own stream.
mf_status after_advance(mf_server* sv, Job* j, Slot& sl) {
  if (j->eng.phase == PH_DONE) return job_finish_enqueue(sv, j, sl, j->slot);
  // idle: the mirrored scalars are current and nothing is in flight on the request's stream
  if (j->eng.idle && !j->cancel) {
    j->batch_ready = true;
    return MF_OK;
  }
  return cuda_check(cudaEventRecord(sl.ev, sl.s), "event record");
}

// One batched CG iteration of a class's planned composition as a CUDA graph (apply, alpha,
// update, direction), launched chunk times per chunk.  A graph of one iteration keeps the
// re-capture after a membership change short (a handful of launches instead of a chunk's
// worth); an existing executable graph is updated in place when the new one differs only in
// parameters (launch sizes), else rebuilt.
mf_status capture_iteration(BatchClass* c) {
  mf_status st = cuda_check(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal), "batch capture");
  if (st) return st;
  const mf_status cst = batch_iteration(c->plan, c->s);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->s, &g);
  if (cst || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cst ? cst : cuda_check(ce, "batch capture end");
  }
  if (c->exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(c->exec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(c->exec);
      c->exec = nullptr;
    }
  }
  if (!c->exec) st = cuda_check(cudaGraphInstantiate(&c->exec, g, 0), "batch graph instantiate");
  cudaGraphDestroy(g);
  c->exec_current = st == MF_OK;
  return st;
}

// A chunk: chunk launches of the iteration graph, then the members' CG states gathered and
// copied to the pinned mirror.
mf_status launch_chunk(BatchClass* c, int chunk, int n) {
  mf_status st = MF_OK;
  for (int it = 0; it < chunk && st == MF_OK; ++it) st = cuda_check(cudaGraphLaunch(c->exec, c->s), "batch launch");
  CgState* states_dev = reinterpret_cast<CgState*>(c->dev + c->states_off);
  if (!st) st = batch_gather_states(c->plan, states_dev, c->s);
  if (!st)
    st = cuda_check(cudaMemcpyAsync(c->host + c->states_off, states_dev, sizeof(CgState) * (size_t)n,
                                    cudaMemcpyDeviceToHost, c->s), "batch states D2H");
  return st;
}

// Chunks of batched CG iterations: collect finished ones, then start new ones.
bool run_batches(mf_server* sv) {
  bool progressed = false;
  for (BatchClass* c : sv->classes) {
    if (!c->running) continue;
    const cudaError_t q = cudaEventQuery(c->ev);
    if (q == cudaErrorNotReady) continue;
    progressed = true;
    c->running = false;
    const CgState* hs = reinterpret_cast<const CgState*>(c->host + c->states_off);
    for (size_t k = 0; k < c->members.size(); ++k) {
      Job* j = c->members[k];
      Slot& sl = sv->slots[j->slot];
      j->in_batch = false;
      if (q != cudaSuccess) {
        job_fail(sv, j, &sl, cuda_check(q, "batch stream"));
        continue;
      }
      j->eng.hm->st = hs[k];
      if (++j->steps > j->max_steps) {
        job_fail(sv, j, &sl, set_error(MF_ERR_TIMEOUT, "request %llu made no progress", (unsigned long long)j->ticket));
        continue;
      }
      j->eng.cancel = j->cancel;
      mf_status st = engine_advance(&j->eng);
      if (!st) st = after_advance(sv, j, sl);
      if (st) job_fail(sv, j, &sl, st);
    }
    c->members.clear();
  }
  // group the waiting requests by class
  std::vector<std::pair<BatchClass*, Job*>> ready;
  for (auto& sl : sv->slots) {
    Job* j = sl.job;
    if (!j || !j->batch_ready || j->in_batch) continue;
    BatchClass* c = class_of(sv, j);
    if (!c) { // no batch buffers: run this request's own chunks
      j->batch_ready = false;
      j->eng.external = false;
      mf_status st = engine_advance(&j->eng);
      if (!st) st = after_advance(sv, j, sl);
      if (st) job_fail(sv, j, &sl, st);
      progressed = true;
      continue;
    }
    ready.emplace_back(c, j);
  }
  for (BatchClass* c : sv->classes) {
    if (c->running) continue;
    std::vector<Job*> mem;
    for (auto& pr : ready)
      if (pr.first == c && (int)mem.size() < c->cap) mem.push_back(pr.second);
    if (mem.empty()) continue;
    progressed = true;
    std::vector<uint64_t> tickets;
    for (Job* j : mem) tickets.push_back(j->ticket);
    mf_status st = MF_OK;
    if (tickets != c->planned) {
      std::vector<BatchMember> bm;
      for (Job* j : mem) bm.push_back(engine_batch_member(&j->eng));
      st = batch_plan_build(&c->plan, bm.data(), (int)bm.size(), c->elem, c->dev, c->host, c->s);
      c->planned = st ? std::vector<uint64_t>() : tickets;
      c->exec_current = false;
    }
    if (!st && !c->exec_current) st = capture_iteration(c);
    if (!st) st = launch_chunk(c, mem[0]->eng.chunk, (int)mem.size());
    if (!st) st = cuda_check(cudaEventRecord(c->ev, c->s), "batch event");
    if (st) {
      cudaStreamSynchronize(c->s);
      c->planned.clear();
      c->exec_current = false;
      for (Job* j : mem) {
        j->batch_ready = false;
        job_fail(sv, j, &sv->slots[j->slot], st);
      }
      continue;
    }
    for (Job* j : mem) {
      j->batch_ready = false;
      j->in_batch = true;
    }
    c->members = mem;
    c->running = true;
  }
  return progressed;
}

void scheduler(mf_server* sv) {
  cudaSetDevice(sv->device);
  const int nslot = (int)sv->slots.size();
  while (!sv->stop.load()) {
    bool progressed = false;
    // admission: arrival order, skipping requests that do not fit yet
    std::vector<std::pair<Job*, int>> admitted;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        int free_slot = -1;
        for (int i = 0; i < nslot; ++i)
          if (!sv->slots[i].job) { free_slot = i; break; }
        if (free_slot < 0) break;
        Job* j = *it;
        if (j->cancel) {
          j->status = MF_ERR_CANCELLED;
          j->t_done = now_s(sv);
          j->stage = ST_DONE;
          job_free_host(j);
          sv->completed += 1;
          it = sv->pending.erase(it);
          sv->cv.notify_all();
          continue;
        }
        char* m = sv->arena.alloc(j->bytes);
        if (!m) { ++it; continue; }
        j->mem = m;
        j->slot = free_slot;
        j->t_admit = now_s(sv);
        sv->slots[free_slot].job = j;
        sv->admitted += 1;
        admitted.emplace_back(j, free_slot);
        it = sv->pending.erase(it);
      }
    }
    for (auto& pr : admitted) {
      Slot& sl = sv->slots[pr.second];
      mf_status st = job_start(sv, pr.first, sl, &sv->mirrors[pr.second]);
      if (st) job_fail(sv, pr.first, &sl, st);
      progressed = true;
    }
    // progress of active requests
    for (int i = 0; i < nslot; ++i) {
      Slot& sl = sv->slots[i];
      Job* j = sl.job;
      if (!j || j->in_batch) continue;
      if (j->batch_ready) {
        if (!j->cancel) continue; // waits for its class's next chunk
        j->batch_ready = false;   // cancelled while waiting: finish on its own stream
        j->eng.cancel = true;
        mf_status st = engine_advance(&j->eng);
        if (!st) st = after_advance(sv, j, sl);
        if (st) job_fail(sv, j, &sl, st);
        progressed = true;
        continue;
      }
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      if (q != cudaSuccess) { job_fail(sv, j, &sl, cuda_check(q, "request stream")); continue; }
      mf_status st = MF_OK;
      if (j->stage == ST_SOLVING) {
        j->eng.cancel = j->cancel;
        if (++j->steps > j->max_steps) {
          job_fail(sv, j, &sl, set_error(MF_ERR_TIMEOUT, "request %llu made no progress", (unsigned long long)j->ticket));
          continue;
        }
        st = engine_advance(&j->eng);
        if (!st) st = after_advance(sv, j, sl);
      } else if (j->stage == ST_FINISHING) {
        job_retire(sv, j, sl, i);
        continue;
      }
      if (st) job_fail(sv, j, &sl, st);
    }
    if (run_batches(sv)) progressed = true;
    if (!progressed) {
      std::unique_lock<std::mutex> lk(sv->mu);
      bool idle = true;
      for (int i = 0; i < nslot; ++i)
        if (sv->slots[i].job) { idle = false; break; }
      if (idle && sv->pending.empty())
        sv->cv.wait_for(lk, std::chrono::milliseconds(2));
      else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    }
  }
}

} // namespace
} // namespace mf

using namespace mf;

extern "C" {

mf_status mf_server_create(const mf_server_config* cfg, void* arena_dev, size_t arena_bytes, mf_server** out) {
  if (!out) return set_error(MF_ERR_ARG, "mf_server_create: out is NULL");
  *out = nullptr;
  if (!arena_dev || arena_bytes < 4096) return set_error(MF_ERR_ARG, "mf_server_create: arena missing or too small");
  if (reinterpret_cast<uintptr_t>(arena_dev) & 255) return set_error(MF_ERR_ARG, "mf_server_create: arena alignment");
  if (cfg && (cfg->mixed_restart < 0 || cfg->mixed_restart > 1 || cfg->inner_rtol < 0.0 || cfg->inner_rtol >= 1.0))
    return set_error(MF_ERR_ARG, "mf_server_create: bad mixed_restart or inner_rtol");
  mf_server* sv = new (std::nothrow) mf_server;
  if (!sv) return set_error(MF_ERR_OOM, "mf_server_create: host allocation failed");
  if (cfg) sv->cfg = *cfg;
  if (sv->cfg.max_slots <= 0) sv->cfg.max_slots = 32;
  if (sv->cfg.max_slots > 256) sv->cfg.max_slots = 256;
  if (sv->cfg.queue_capacity <= 0) sv->cfg.queue_capacity = 100000;
  mf_status st = cuda_check(cudaGetDevice(&sv->device), "cudaGetDevice");
  if (st) { delete sv; return st; }
  sv->arena.init(static_cast<char*>(arena_dev), arena_bytes);
  sv->slots.resize(sv->cfg.max_slots);
  if ((st = cuda_check(cudaMallocHost(&sv->mirrors, sizeof(HostMirror) * sv->cfg.max_slots), "pinned mirrors")) ||
      (st = cuda_check(cudaMallocHost(&sv->l2_host, sizeof(double) * sv->cfg.max_slots), "pinned l2"))) {
    if (sv->mirrors) cudaFreeHost(sv->mirrors);
    delete sv;
    return st;
  }
  std::memset(sv->mirrors, 0, sizeof(HostMirror) * sv->cfg.max_slots);
  for (auto& sl : sv->slots) {
    if ((st = cuda_check(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking), "slot stream"))) break;
    if ((st = cuda_check(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming), "slot event"))) break;
  }
  if (st) {
    for (auto& sl : sv->slots) {
      if (sl.s) cudaStreamDestroy(sl.s);
      if (sl.ev) cudaEventDestroy(sl.ev);
    }
    cudaFreeHost(sv->mirrors);
    cudaFreeHost(sv->l2_host);
    delete sv;
    return st;
  }
  sv->t0 = std::chrono::steady_clock::now();
  sv->th = std::thread(scheduler, sv);
  *out = sv;
  return MF_OK;
}

mf_status mf_batch_submit(mf_server* sv, const mf_request* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return set_error(MF_ERR_ARG, "mf_batch_submit: NULL argument");
  if (req->rhs != MF_RHS_MANUFACTURED && req->rhs != MF_RHS_RANDOM)
    return set_error(MF_ERR_ARG, "mf_batch_submit: unknown rhs kind %d", req->rhs);
  if (!(req->rtol >= 0.0) || req->maxit <= 0) return set_error(MF_ERR_ARG, "mf_batch_submit: bad rtol/maxit");
  Job* j = new (std::nothrow) Job;
  if (!j) return set_error(MF_ERR_OOM, "mf_batch_submit: host allocation failed");
  j->req = *req;
  mf_status st = job_prepare(sv, j);
  if (st) {
    job_free_host(j);
    delete j;
    return st;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if ((int)sv->pending.size() >= sv->cfg.queue_capacity) {
    job_free_host(j);
    delete j;
    return set_error(MF_ERR_BUSY, "mf_batch_submit: queue full");
  }
  j->ticket = sv->next_ticket++;
  j->t_submit = now_s(sv);
  sv->pending.push_back(j);
  sv->jobs[j->ticket] = j;
  *ticket = j->ticket;
  sv->cv.notify_all();
  return MF_OK;
}

mf_status mf_batch_poll(mf_server* sv, uint64_t ticket, mf_result* res) {
  if (!sv || !res) return set_error(MF_ERR_ARG, "mf_batch_poll: NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return set_error(MF_ERR_ARG, "mf_batch_poll: unknown ticket %llu", (unsigned long long)ticket);
  Job* j = it->second;
  std::memset(res, 0, sizeof(*res));
  res->t_submit = j->t_submit;
  res->t_admit = j->t_admit;
  res->n_cellwise = j->info.n_cellwise;
  res->n_unique = j->info.n_unique;
  res->device_bytes = j->bytes;
  if (j->stage != ST_DONE) {
    res->status = MF_ERR_BUSY;
    return MF_ERR_BUSY;
  }
  res->status = j->status;
  res->iterations = j->eng.total_it;
  res->outer_iterations = j->req.mixed ? j->eng.outer : 1;
  res->rel_residual = j->eng.rel;
  res->l2_error = j->l2;
  res->t_done = j->t_done;
  res->latency = j->t_done - j->t_submit;
  sv->jobs.erase(it);
  delete j;
  return MF_OK;
}

mf_status mf_batch_cancel(mf_server* sv, uint64_t ticket) {
  if (!sv) return set_error(MF_ERR_ARG, "mf_batch_cancel: NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return set_error(MF_ERR_ARG, "mf_batch_cancel: unknown ticket");
  it->second->cancel = true;
  return MF_OK;
}

mf_status mf_server_drain(mf_server* sv, double timeout_s) {
  if (!sv) return set_error(MF_ERR_ARG, "mf_server_drain: NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  auto busy = [&]() {
    if (!sv->pending.empty()) return true;
    for (auto& sl : sv->slots)
      if (sl.job) return true;
    return false;
  };
  while (busy()) {
    if (sv->cv.wait_until(lk, deadline) == std::cv_status::timeout && busy())
      return set_error(MF_ERR_TIMEOUT, "mf_server_drain: still busy after %.3f s", timeout_s);
  }
  return MF_OK;
}

mf_status mf_server_stats(mf_server* sv, mf_server_stats_t* out) {
  if (!sv || !out) return set_error(MF_ERR_ARG, "mf_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->pending = (int64_t)sv->pending.size();
  int active = 0;
  for (auto& sl : sv->slots)
    if (sl.job) ++active;
  out->active = active;
  out->admitted = sv->admitted;
  out->completed = sv->completed;
  out->arena_bytes = sv->arena.size();
  out->arena_used = sv->arena.used();
  out->arena_peak = sv->arena.peak();
  return MF_OK;
}

void mf_server_destroy(mf_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto& kv : sv->jobs) kv.second->cancel = true;
  }
  sv->stop.store(true);
  sv->cv.notify_all();
  if (sv->th.joinable()) sv->th.join();
  for (BatchClass* c : sv->classes) class_destroy(sv, c);
  sv->classes.clear();
  for (auto& sl : sv->slots) {
    if (sl.s) cudaStreamSynchronize(sl.s);
    if (sl.job) engine_release(&sl.job->eng);
  }
  for (auto& kv : sv->jobs) {
    job_free_host(kv.second);
    delete kv.second;
  }
  for (auto& sl : sv->slots) {
    if (sl.s) cudaStreamDestroy(sl.s);
    if (sl.ev) cudaEventDestroy(sl.ev);
  }
  cudaFreeHost(sv->mirrors);
  cudaFreeHost(sv->l2_host);
  delete sv;
}

} // extern "C"
