// Serving: continuous batching of submitted simulations on one GPU.
//
// A host worker thread owns every running simulation.  Submitted requests
// wait in submission order and are admitted as soon as their state
// (pic_query's arena size) fits the budget next to the running ones; a
// request that fits may go ahead of earlier ones that do not, unless the
// oldest waiting request has waited longer than kHeadWait, in which case
// memory is left to free up for it.  Each admitted simulation keeps all of
// its state on the device until it finishes, in a range of the server's
// own device memory (DeviceArena): chunks reserved with cudaMalloc as
// requests need them, up to the budget, and kept until the server is
// destroyed, so admitting and finishing requests neither allocates nor
// frees device memory (cudaFree would wait for the whole device).  The running simulations with at least a quantum of steps left
// advance together from one CUDA graph (pic_batch_*), rebuilt only when that
// set changes; one with fewer steps left takes them alone.  A finished
// request's FP64 diagnostics (and, if asked, its final fields) are kept until
// its ticket is polled, and its device memory is released at once.
//
// Built only on the public C ABI of the simulation (include/pic.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pic.h"

namespace pg_internal {
void set_last_error(const std::string &msg);  // pic_last_error() of this thread
}  // namespace pg_internal

namespace {

using Clock = std::chrono::steady_clock;

int serve_fail(int code, const std::string &msg) {
  pg_internal::set_last_error(msg);
  return code;
}

struct Request {
  long long ticket = 0;
  pic_grid grid{};
  std::vector<pic_layer> layers;
  pic_pulse pulse{};
  uint64_t seed = 0;
  long long steps = 0;
  int n_bins = 0;
  double e_min = 0.0, e_max = 0.0;
  double *fields_out = nullptr;  // caller-owned, 15 * nfield doubles
  unsigned long long need = 0;   // arena bytes
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  // result
  bool done = false;
  int status = PIC_OK;
  std::string message;
  pic_diag diag{};
  std::vector<double> spectrum;
};

struct Running {
  std::shared_ptr<Request> req;
  pic_handle h = nullptr;
  cudaStream_t stream = nullptr;
  char *arena = nullptr;  // the request's range of the server's device memory
  long long left = 0;
};

// A waiting request older than this blocks the admission of later ones.
constexpr double kHeadWait = 1.0;  // seconds

// Device memory of a server: chunks of at least kChunk bytes (or one
// request's arena) reserved with cudaMalloc when no free range fits, never
// more than the budget in total, carved first-fit into 256-byte aligned
// ranges and coalesced when released.
class DeviceArena {
 public:
  static constexpr size_t kAlign = 256;
  static constexpr size_t kChunk = size_t(16) << 30;

  explicit DeviceArena(unsigned long long budget) : budget_(budget) {}
  ~DeviceArena() {
    for (Chunk &c : chunks_) cudaFree(c.base);
  }

  // A range of n bytes, or nullptr when none is free now (and no chunk may
  // or can be reserved).
  char *alloc(size_t n) {
    n = (n + kAlign - 1) / kAlign * kAlign;
    for (Chunk &c : chunks_)
      for (auto it = c.free.begin(); it != c.free.end(); ++it)
        if (it->second >= n) {
          const size_t off = it->first, len = it->second;
          c.free.erase(it);
          if (len > n) c.free[off + n] = len - n;
          return c.base + off;
        }
    if (reserved_ + n > budget_) return nullptr;
    size_t size = std::max(n, std::min<size_t>(kChunk, (size_t)(budget_ - reserved_)));
    char *base = nullptr;
    if (cudaMalloc((void **)&base, size) != cudaSuccess) {
      (void)cudaGetLastError();
      size = n;
      if (cudaMalloc((void **)&base, size) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
      }
    }
    Chunk c;
    c.base = base;
    c.size = size;
    if (size > n) c.free[n] = size - n;
    chunks_.push_back(std::move(c));
    reserved_ += size;
    return base;
  }

  void release(char *p, size_t n) {
    n = (n + kAlign - 1) / kAlign * kAlign;
    for (Chunk &c : chunks_) {
      if (p < c.base || p >= c.base + c.size) continue;
      size_t off = (size_t)(p - c.base);
      auto next = c.free.lower_bound(off);
      if (next != c.free.end() && off + n == next->first) {
        n += next->second;
        next = c.free.erase(next);
      }
      if (next != c.free.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
          prev->second += n;
          return;
        }
      }
      c.free[off] = n;
      return;
    }
  }

 private:
  struct Chunk {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free;  // offset -> length
  };
  std::vector<Chunk> chunks_;
  unsigned long long budget_;
  unsigned long long reserved_ = 0;
};

}  // namespace

struct pic_server_ctx {
  unsigned long long budget = 0;
  int quantum = 32;
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  long long next_ticket = 1;
  std::deque<std::shared_ptr<Request>> waiting;
  std::map<long long, std::shared_ptr<Request>> all;  // submitted and not yet collected
  std::thread worker;
  // worker-only state
  std::vector<Running> running;
  unsigned long long used = 0;
  std::unique_ptr<DeviceArena> mem;
  pic_batch batch = nullptr;
  std::vector<pic_handle> batch_members;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void run();
  void loop();
  void finish(Running &r, int status, const std::string &msg);
  void admit();
  void rebatch();
};

void pic_server_ctx::finish(Running &r, int status, const std::string &msg) {
  Request &q = *r.req;
  if (status == PIC_OK) {
    std::memset(&q.diag, 0, sizeof(q.diag));
    q.spectrum.assign(q.n_bins > 0 ? q.n_bins : 1, 0.0);
    q.diag.n_bins = q.n_bins;
    q.diag.e_min_eV = q.e_min;
    q.diag.e_max_eV = q.e_max;
    const int box[6] = {0, q.grid.nx, 0, q.grid.ny, 0, q.grid.nz};
    std::memcpy(q.diag.region, box, sizeof(box));
    q.diag.spectrum = q.spectrum.data();
    status = pic_diagnostics(r.h, &q.diag);
    if (status == PIC_OK && q.fields_out) status = pic_get_fields(r.h, q.fields_out);
  }
  const std::string m = status == PIC_OK ? std::string() : (msg.empty() ? pic_last_error() : msg);
  if (r.h) pic_destroy(r.h);
  // the handle's stream has no work left (every finish follows a sync or a
  // failed create), so the range is free for the next request
  if (r.stream) cudaStreamDestroy(r.stream);
  if (r.arena) mem->release(r.arena, q.need);
  r.h = nullptr;
  r.stream = nullptr;
  r.arena = nullptr;
  used -= q.need;
  std::lock_guard<std::mutex> lk(mu);
  q.status = status;
  q.message = m;
  q.t_done = now();
  q.done = true;
  cv_done.notify_all();
}

// Admit waiting requests in submission order while they fit the budget and
// a free range of the server's memory; later requests may pass one that does
// not fit, unless the oldest waiting request has waited kHeadWait or longer.
void pic_server_ctx::admit() {
  for (size_t idx = 0;;) {
    std::shared_ptr<Request> q;
    char *arena = nullptr;
    {
      std::lock_guard<std::mutex> lk(mu);
      if (idx >= waiting.size()) return;
      if (idx > 0 && now() - waiting.front()->t_submit >= kHeadWait) return;
      q = waiting[idx];
      if (used + q->need <= budget) arena = mem->alloc(q->need);
      if (!arena) {
        if (running.empty() && used == 0) {
          // nothing holds memory and the range still cannot be had: the
          // device itself is out of memory for this request
          waiting.erase(waiting.begin() + (long)idx);
          q->status = PIC_ENOMEM;
          q->message = "no device memory for the request's state";
          q->t_admit = q->t_done = now();
          q->done = true;
          cv_done.notify_all();
          continue;
        }
        ++idx;
        continue;
      }
      waiting.erase(waiting.begin() + (long)idx);
    }
    Running r;
    r.req = q;
    r.left = q->steps;
    r.arena = arena;
    used += q->need;
    q->t_admit = now();
    int rc = PIC_OK;
    std::string msg;
    cudaError_t e = cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      rc = PIC_ECUDA;
      msg = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      r.stream = nullptr;
    } else {
      pic_material m;
      std::memset(&m, 0, sizeof(m));
      m.n_layers = (int)q->layers.size();
      m.layers = q->layers.data();
      rc = pic_create(&q->grid, &m, &q->pulse, q->seed, r.stream, arena, q->need, &r.h);
    }
    if (rc != PIC_OK || r.left == 0) {
      finish(r, rc, msg);
      continue;
    }
    running.push_back(r);
  }
}

// One graph over the running simulations with at least a quantum left.
void pic_server_ctx::rebatch() {
  std::vector<pic_handle> want;
  for (const Running &r : running)
    if (r.left >= quantum) want.push_back(r.h);
  if (want == batch_members) return;
  if (batch) pic_batch_destroy(batch);
  batch = nullptr;
  batch_members.clear();
  if (want.empty()) return;
  if (pic_batch_create(want.data(), (int)want.size(), nullptr, &batch) == PIC_OK) {
    batch_members = want;
  } else {
    batch = nullptr;  // step them one by one this round
  }
}

// The worker: the loop, and if host memory runs out inside it (the only
// exception it can meet), every request still held fails with PIC_ENOMEM.
void pic_server_ctx::run() {
  try {
    loop();
  } catch (const std::exception &e) {
    const std::string m = std::string("server worker stopped: ") + e.what();
    if (batch) pic_batch_destroy(batch);
    batch = nullptr;
    for (Running &r : running) {
      if (r.h) pic_destroy(r.h);
      if (r.stream) cudaStreamDestroy(r.stream);
    }
    running.clear();
    std::lock_guard<std::mutex> lk(mu);
    stop = true;  // later submits are refused
    for (auto &kv : all)
      if (!kv.second->done) {
        kv.second->status = PIC_ENOMEM;
        kv.second->message = m;
        kv.second->done = true;
      }
    waiting.clear();
    cv_done.notify_all();
  }
}

void pic_server_ctx::loop() {
  cudaSetDevice(device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !waiting.empty() || !running.empty(); });
      if (stop) break;
    }
    admit();
    if (running.empty()) {
      // with nothing running the whole budget is free and submit admits no
      // request larger than it, so the queue is empty here; wait for work
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
      continue;
    }
    rebatch();
    std::vector<int> rc(running.size(), PIC_OK);
    std::vector<std::string> msg(running.size());
    bool batched = false;
    if (batch) {
      if (pic_batch_step(batch, quantum) == PIC_OK) {
        batched = true;
      } else {
        const std::string m = pic_last_error();
        for (size_t q = 0; q < running.size(); ++q)
          if (running[q].left >= quantum) {
            rc[q] = PIC_ECUDA;
            msg[q] = m;
          }
      }
    }
    for (size_t q = 0; q < running.size(); ++q) {
      Running &r = running[q];
      const bool in_batch = batch && r.left >= quantum;
      if (in_batch || rc[q] != PIC_OK) continue;
      const long long n = r.left < quantum ? r.left : quantum;
      rc[q] = pic_step(r.h, (int)n);
      if (rc[q] == PIC_OK) r.left -= n;
      else msg[q] = pic_last_error();
    }
    if (batched) {
      pic_batch_sync(batch);  // member errors are read per member below
      for (Running &r : running)
        if (r.left >= quantum) r.left -= quantum;
    }
    for (size_t q = 0; q < running.size(); ++q)
      if (rc[q] == PIC_OK) {
        rc[q] = pic_sync(running[q].h);
        if (rc[q] != PIC_OK) msg[q] = pic_last_error();
      }
    std::vector<Running> keep;
    for (size_t q = 0; q < running.size(); ++q) {
      if (rc[q] != PIC_OK || running[q].left <= 0) {
        // a member of the graph is about to be destroyed: drop the graph first
        bool member = false;
        for (pic_handle m : batch_members) member |= m == running[q].h;
        if (member) {
          pic_batch_destroy(batch);
          batch = nullptr;
          batch_members.clear();
        }
        finish(running[q], rc[q], msg[q]);
      } else {
        keep.push_back(running[q]);
      }
    }
    running.swap(keep);
  }
  if (batch) pic_batch_destroy(batch);
  batch = nullptr;
  for (Running &r : running) finish(r, PIC_ESTATE, "server destroyed before the request finished");
  running.clear();
  std::lock_guard<std::mutex> lk(mu);
  for (auto &q : waiting) {
    q->status = PIC_ESTATE;
    q->message = "server destroyed before the request was admitted";
    q->done = true;
  }
  waiting.clear();
  cv_done.notify_all();
}

extern "C" {

int pic_serve_create(double budget_bytes, int quantum, pic_server *out) {
  if (!out) return serve_fail(PIC_EINVAL, "null pointer");
  *out = nullptr;
  if (!(budget_bytes >= 1.0 && budget_bytes < 1.8e19) || quantum < 1)
    return serve_fail(PIC_EINVAL, "budget must be >= 1 byte and quantum >= 1");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return serve_fail(PIC_ECUDA, "no CUDA device");
  // no C++ exception may cross the C ABI
  pic_server_ctx *s = nullptr;
  try {
    s = new pic_server_ctx();
    s->budget = (unsigned long long)budget_bytes;
    s->mem.reset(new DeviceArena(s->budget));
    s->quantum = quantum;
    s->device = dev;
    s->t0 = Clock::now();
    s->worker = std::thread([s] { s->run(); });
  } catch (const std::exception &e) {
    delete s;
    return serve_fail(PIC_ENOMEM, std::string("cannot start the server: ") + e.what());
  }
  *out = s;
  return PIC_OK;
}

int pic_serve_submit(pic_server s, const pic_grid *grid, const pic_material *mat,
                     const pic_pulse *pulse, uint64_t seed, long long n_steps, int n_bins,
                     double e_min_eV, double e_max_eV, double *fields_out, long long *ticket) {
  if (!s || !grid || !mat || !pulse || !ticket) return serve_fail(PIC_EINVAL, "null pointer");
  if (n_steps < 0) return serve_fail(PIC_EINVAL, "negative step count");
  if (n_bins < 0 || n_bins > 65536 || (n_bins > 0 && !(e_max_eV > e_min_eV)))
    return serve_fail(PIC_EINVAL, "bad spectrum request");
  pic_info info;
  const int rc = pic_query(grid, mat, pulse, &info);
  if (rc != PIC_OK) return serve_fail(rc, pic_last_error());
  if ((unsigned long long)info.arena_bytes > s->budget)
    return serve_fail(PIC_ENOMEM, "the request alone needs more than the server's budget");
  std::shared_ptr<Request> q;
  try {
    q = std::make_shared<Request>();
    q->grid = *grid;
    q->layers.assign(mat->layers, mat->layers + mat->n_layers);
    q->pulse = *pulse;
    q->seed = seed;
    q->steps = n_steps;
    q->n_bins = n_bins;
    q->e_min = e_min_eV;
    q->e_max = e_max_eV;
    q->fields_out = fields_out;
    q->need = (unsigned long long)info.arena_bytes;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return serve_fail(PIC_ESTATE, "server is stopping");
    q->ticket = s->next_ticket++;
    q->t_submit = s->now();
    s->all[q->ticket] = q;
    s->waiting.push_back(q);
  } catch (const std::exception &e) {
    if (q && q->ticket) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->all.erase(q->ticket);
    }
    return serve_fail(PIC_ENOMEM, std::string("cannot queue the request: ") + e.what());
  }
  s->cv_work.notify_one();
  *ticket = q->ticket;
  return PIC_OK;
}

int pic_serve_poll(pic_server s, long long ticket, int wait_ms, int *done, pic_diag *diag,
                   double times[3]) {
  if (!s || !done) return serve_fail(PIC_EINVAL, "null pointer");
  *done = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return serve_fail(PIC_EINVAL, "unknown ticket");
  std::shared_ptr<Request> q = it->second;
  if (!q->done && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return q->done; });
  if (!q->done) return PIC_OK;
  if (diag) {
    if (q->status == PIC_OK && q->n_bins > 0 && (!diag->spectrum || diag->n_bins < q->n_bins))
      return serve_fail(PIC_EINVAL, "diag needs a spectrum buffer of the submitted n_bins");
    double *spec = diag->spectrum;
    if (q->status == PIC_OK) {
      *diag = q->diag;
      diag->spectrum = spec;
      if (q->n_bins > 0) std::memcpy(spec, q->spectrum.data(), q->n_bins * sizeof(double));
    }
  }
  if (times) {
    times[0] = q->t_submit;
    times[1] = q->t_admit;
    times[2] = q->t_done;
  }
  *done = 1;
  s->all.erase(it);
  if (q->status != PIC_OK) return serve_fail(q->status, q->message);
  return PIC_OK;
}

int pic_serve_destroy(pic_server s) {
  if (!s) return PIC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
  return PIC_OK;
}

}  // extern "C"
