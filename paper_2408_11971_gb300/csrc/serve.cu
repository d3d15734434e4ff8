// serve.cu — continuous batching of operator requests over resident
// compressed streams (hoszp_server_*, declared in include/hoszp.h).
//
// One scheduling thread owns every GPU call. It admits requests in arrival
// order into free slots when the output arena can hold their result (see
// serve_arena.h), launches each on its slot's own stream with the slot's own
// context, and notices completions through events, so requests that arrive
// while others run start as soon as a slot and memory free up and their
// kernels overlap on the device. Results, sizes and the context status of a
// request come back through pinned host memory without synchronizing.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "hz_common.cuh"
#include "serve_arena.h"

namespace hz {
int* ctx_status_word(hoszp_ctx* ctx);           // api.cu
size_t ctx_workspace_bytes(const hoszp_ctx* ctx);
void ctx_limit_sms(hoszp_ctx* ctx, int sms);
}  // namespace hz

using namespace hz;

namespace {

struct SrvStream {
  const void* d;
  size_t bytes;
  uint64_t n, nb;
};

struct SrvReq {
  hoszp_request r;
  uint64_t arrival_us;
  SrvStream sa, sb;  // copies taken at submission (registration may grow the table meanwhile)
};

struct HostRes {  // pinned, one per slot
  double value;
  unsigned long long bytes;
  int status;
  int pad;
};

struct Slot {
  hoszp_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  SrvReq req{};
  uint64_t off = ~0ull;
  uint64_t start_us = 0;
  double* d_val = nullptr;
  unsigned long long* d_bytes = nullptr;
  HostRes* h = nullptr;
};

uint64_t out_bound(int op, const SrvStream& a, const SrvStream* b, double s) {
  switch (op) {
    case HOSZP_OP_NEGATE:
    case HOSZP_OP_ADD_SCALAR:
      return a.bytes;
    case HOSZP_OP_MUL_SCALAR: {
      // a block's rate grows by at most e bits (|2 eps rho| <= 2|s|), constant blocks stay
      const double e = std::ceil(std::log2(2.0 * std::fabs(s) + 1.0)) + 1.0;
      const uint64_t bound = a.bytes + 8ull * a.nb * (uint64_t)e + 16;
      const uint64_t worst = hoszp_compress_bound(a.n);
      return bound < worst ? bound : worst;
    }
    case HOSZP_OP_ADD:
    case HOSZP_OP_SUB:
      return a.bytes + (b ? b->bytes : 0);
    case HOSZP_OP_DECOMPRESS:
      return 4 * a.n;
    default:
      return 0;
  }
}

}  // namespace

struct hoszp_server {
  int device = 0;
  uint64_t max_n = 0;
  std::vector<Slot> slots;
  void* arena_mem = nullptr;
  void* scratch_mem = nullptr;
  HostRes* host_res = nullptr;
  uint64_t workspace_bytes = 0;
  serve::Arena arena;
  std::vector<SrvStream> streams;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<SrvReq> pending;
  std::deque<hoszp_completion> done;
  std::thread th;
  std::atomic<bool> stop{false};
  std::chrono::steady_clock::time_point t0;
  uint64_t submitted = 0, completed = 0, in_flight = 0, max_in_flight = 0;

  uint64_t now() const {
    return (uint64_t)std::chrono::duration_cast<std::chrono::microseconds>(
               std::chrono::steady_clock::now() - t0)
        .count();
  }
  static uint64_t need(const SrvReq& q) {
    const bool two = q.r.op == HOSZP_OP_ADD || q.r.op == HOSZP_OP_SUB;
    return out_bound(q.r.op, q.sa, two ? &q.sb : nullptr, q.r.scalar);
  }
  void complete(const SrvReq& q, int status, double value, void* out, uint64_t out_bytes,
                uint64_t start_us) {
    hoszp_completion c;
    std::memset(&c, 0, sizeof(c));
    c.tag = q.r.tag;
    c.op = q.r.op;
    c.status = status;
    c.value = value;
    c.d_out = out;
    c.out_bytes = out_bytes;
    c.arrival_us = q.arrival_us;
    c.start_us = start_us;
    c.done_us = now();
    {
      std::lock_guard<std::mutex> lk(mu);
      done.push_back(c);
      completed++;
    }
    cv_done.notify_all();
  }
  // Launches q on slot k (its output block at `off`, ~0 for none). Scheduler thread only.
  void launch(int k, const SrvReq& q, uint64_t off) {
    Slot& sl = slots[k];
    const SrvStream& a = q.sa;
    uint8_t* out = off == ~0ull ? nullptr : static_cast<uint8_t*>(arena_mem) + off;
    const uint64_t cap = off == ~0ull ? 0 : need(q);
    const hoszp_stream_t st = reinterpret_cast<hoszp_stream_t>(sl.st);
    unsigned long long* ob = sl.d_bytes;
    int rc = HOSZP_OK;
    switch (q.r.op) {
      case HOSZP_OP_MEAN: rc = hoszp_mean(sl.ctx, a.d, a.bytes, sl.d_val, st); break;
      case HOSZP_OP_VAR: rc = hoszp_var(sl.ctx, a.d, a.bytes, sl.d_val, st); break;
      case HOSZP_OP_NEGATE: rc = hoszp_negate(sl.ctx, a.d, a.bytes, out, cap, (uint64_t*)ob, st); break;
      case HOSZP_OP_ADD_SCALAR:
        rc = hoszp_add_scalar(sl.ctx, a.d, a.bytes, q.r.scalar, out, cap, (uint64_t*)ob, st);
        break;
      case HOSZP_OP_MUL_SCALAR:
        rc = hoszp_mul_scalar(sl.ctx, a.d, a.bytes, q.r.scalar, out, cap, (uint64_t*)ob, st);
        break;
      case HOSZP_OP_ADD:
      case HOSZP_OP_SUB: {
        const SrvStream& b = q.sb;
        rc = (q.r.op == HOSZP_OP_ADD ? hoszp_add : hoszp_sub)(sl.ctx, a.d, a.bytes, b.d, b.bytes, out,
                                                              cap, (uint64_t*)ob, st);
        break;
      }
      case HOSZP_OP_DECOMPRESS:
        rc = hoszp_decompress(sl.ctx, a.d, a.bytes, reinterpret_cast<float*>(out), a.n, st);
        break;
      default: rc = HOSZP_ERR_ARG;
    }
    const uint64_t t = now();
    if (rc != HOSZP_OK) {  // nothing of it runs on the device
      if (off != ~0ull) {
        std::lock_guard<std::mutex> lk(mu);
        arena.release(off);
      }
      complete(q, rc, 0.0, nullptr, 0, t);
      return;
    }
    int* stw = ctx_status_word(sl.ctx);
    cudaMemcpyAsync(&sl.h->value, sl.d_val, sizeof(double), cudaMemcpyDeviceToHost, sl.st);
    cudaMemcpyAsync(&sl.h->bytes, sl.d_bytes, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                    sl.st);
    cudaMemcpyAsync(&sl.h->status, stw, sizeof(int), cudaMemcpyDeviceToHost, sl.st);
    cudaMemsetAsync(stw, 0, sizeof(int), sl.st);
    if (cudaEventRecord(sl.ev, sl.st) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(sl.st);
    }
    sl.busy = true;
    sl.req = q;
    sl.off = off;
    sl.start_us = t;
    std::lock_guard<std::mutex> lk(mu);
    in_flight++;
    if (in_flight > max_in_flight) max_in_flight = in_flight;
  }
  // A finished slot: its result into a completion, the unused output tail back.
  void finish(int k) {
    Slot& sl = slots[k];
    const SrvReq q = sl.req;
    const int op = q.r.op;
    int status = sl.h->status;
    double value = 0.0;
    void* out = nullptr;
    uint64_t ob = 0;
    if (op == HOSZP_OP_MEAN || op == HOSZP_OP_VAR) {
      value = sl.h->value;
    } else if (status == HOSZP_OK) {
      out = static_cast<uint8_t*>(arena_mem) + sl.off;
      ob = op == HOSZP_OP_DECOMPRESS ? 4 * q.sa.n : sl.h->bytes;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      if (sl.off != ~0ull) {
        if (out) arena.shrink(sl.off, ob);
        else arena.release(sl.off);
      }
      in_flight--;
    }
    sl.busy = false;
    sl.off = ~0ull;
    complete(q, status, value, out, ob, sl.start_us);
  }
  void loop() {
    cudaSetDevice(device);
    for (;;) {
      bool progress = false;
      for (size_t k = 0; k < slots.size(); k++) {
        if (!slots[k].busy) continue;
        const cudaError_t e = cudaEventQuery(slots[k].ev);
        if (e == cudaSuccess) {
          finish((int)k);
          progress = true;
        } else if (e != cudaErrorNotReady) {
          cudaGetLastError();
          slots[k].h->status = HOSZP_ERR_CUDA;
          finish((int)k);
          progress = true;
        }
      }
      for (;;) {  // admissions
        int free_slot = -1;
        for (size_t k = 0; k < slots.size(); k++)
          if (!slots[k].busy) {
            free_slot = (int)k;
            break;
          }
        if (free_slot < 0) break;
        SrvReq q;
        uint64_t off = ~0ull;
        {
          std::lock_guard<std::mutex> lk(mu);
          const long i = serve::pick_next(pending, now(), arena,
                                          [](const SrvReq& x) { return need(x); }, &off);
          if (i < 0) break;
          q = pending[(size_t)i];
          pending.erase(pending.begin() + i);
        }
        launch(free_slot, q, off);
        progress = true;
      }
      bool idle;
      {
        std::lock_guard<std::mutex> lk(mu);
        idle = in_flight == 0;
        if (stop.load() && idle && pending.empty()) break;
      }
      if (!progress) {
        std::unique_lock<std::mutex> lk(mu);
        if (idle && (pending.empty() || pending.front().arrival_us > now() + 50)) {
          const uint64_t t = pending.empty() ? 1000 : pending.front().arrival_us - now();
          cv_work.wait_for(lk, std::chrono::microseconds(t < 1000 ? t : 1000));
        } else {
          lk.unlock();
          std::this_thread::yield();
        }
      }
    }
  }
  void release_all() {
    for (Slot& sl : slots) {
      if (sl.ev) cudaEventDestroy(sl.ev);
      if (sl.st) cudaStreamDestroy(sl.st);
      if (sl.ctx) hoszp_ctx_destroy(sl.ctx);
    }
    slots.clear();
    if (arena_mem) cudaFree(arena_mem);
    if (scratch_mem) cudaFree(scratch_mem);
    if (host_res) cudaFreeHost(host_res);
    arena_mem = scratch_mem = nullptr;
    host_res = nullptr;
  }
};

extern "C" {

int hoszp_server_create(int device, uint32_t nslots, uint64_t budget, uint64_t max_n,
                        uint32_t sms_per_request, hoszp_server** out) {
  if (!out) return HOSZP_ERR_ARG;
  *out = nullptr;
  if (nslots < 1 || nslots > 64 || max_n < 1 || max_n > (1ull << 40)) return HOSZP_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HOSZP_ERR_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  hoszp_server* s = new (std::nothrow) hoszp_server();
  if (!s) return HOSZP_ERR_CUDA;
  s->device = device;
  s->max_n = max_n;
  s->t0 = std::chrono::steady_clock::now();
  int rc = HOSZP_OK;
  s->slots.resize(nslots);
  const size_t scratch = 256 * (size_t)nslots;
  if (cudaMalloc(&s->scratch_mem, scratch) != cudaSuccess ||
      cudaMallocHost((void**)&s->host_res, sizeof(HostRes) * nslots) != cudaSuccess) {
    cudaGetLastError();
    rc = HOSZP_ERR_CUDA;
  }
  s->workspace_bytes = scratch;
  for (uint32_t k = 0; rc == HOSZP_OK && k < nslots; k++) {
    Slot& sl = s->slots[k];
    if ((rc = hoszp_ctx_create(&sl.ctx, device)) != HOSZP_OK) break;
    if ((rc = hoszp_ctx_reserve(sl.ctx, max_n)) != HOSZP_OK) break;
    ctx_limit_sms(sl.ctx, (int)sms_per_request);
    s->workspace_bytes += ctx_workspace_bytes(sl.ctx);
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      rc = HOSZP_ERR_CUDA;
      break;
    }
    uint8_t* base = static_cast<uint8_t*>(s->scratch_mem) + 256 * (size_t)k;
    sl.d_val = reinterpret_cast<double*>(base);
    sl.d_bytes = reinterpret_cast<unsigned long long*>(base + 8);
    sl.h = s->host_res + k;
    std::memset(sl.h, 0, sizeof(HostRes));
  }
  if (rc == HOSZP_OK && s->workspace_bytes + serve::Arena::kAlign > budget) rc = HOSZP_ERR_CAPACITY;
  if (rc == HOSZP_OK) {
    const uint64_t abytes = (budget - s->workspace_bytes) / serve::Arena::kAlign * serve::Arena::kAlign;
    if (cudaMalloc(&s->arena_mem, abytes) != cudaSuccess) {
      cudaGetLastError();
      rc = HOSZP_ERR_CUDA;
    } else {
      s->arena.reset(abytes);
    }
  }
  if (rc != HOSZP_OK) {
    s->release_all();
    delete s;
    cudaSetDevice(prev);
    return rc;
  }
  s->th = std::thread([s]() { s->loop(); });
  cudaSetDevice(prev);
  *out = s;
  return HOSZP_OK;
}

void hoszp_server_destroy(hoszp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.clear();  // queued requests are dropped; those on the device finish
  }
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  s->release_all();
  cudaSetDevice(prev);
  delete s;
}

int hoszp_server_register(hoszp_server* s, const void* d, size_t bytes, uint32_t* id) {
  if (!s || !d || !id || bytes < HOSZP_HEADER_BYTES || ((uintptr_t)d & 15u)) return HOSZP_ERR_ARG;
  hoszp_header h;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  const cudaError_t e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HOSZP_ERR_CUDA;
  }
  if (h.magic != HOSZP_MAGIC || h.version != HOSZP_VERSION || h.block != HOSZP_BLOCK)
    return HOSZP_ERR_FORMAT;
  if (h.n > s->max_n) return HOSZP_ERR_CAPACITY;
  SrvStream st{d, bytes, h.n, nblocks(h.n)};
  std::lock_guard<std::mutex> lk(s->mu);
  s->streams.push_back(st);
  *id = (uint32_t)(s->streams.size() - 1);
  return HOSZP_OK;
}

int hoszp_server_submit(hoszp_server* s, const hoszp_request* r) {
  if (!s || !r || r->op < HOSZP_OP_MEAN || r->op > HOSZP_OP_DECOMPRESS) return HOSZP_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const bool two = r->op == HOSZP_OP_ADD || r->op == HOSZP_OP_SUB;
    if (r->a >= s->streams.size() || (two && r->b >= s->streams.size())) return HOSZP_ERR_ARG;
    if ((r->op == HOSZP_OP_ADD_SCALAR || r->op == HOSZP_OP_MUL_SCALAR) && !std::isfinite(r->scalar))
      return HOSZP_ERR_ARG;
    SrvReq q;
    q.r = *r;
    q.arrival_us = r->arrival_us ? r->arrival_us : s->now();
    q.sa = s->streams[r->a];
    q.sb = two ? s->streams[r->b] : SrvStream{nullptr, 0, 0, 0};
    s->pending.push_back(q);
    s->submitted++;
  }
  s->cv_work.notify_all();
  return HOSZP_OK;
}

int hoszp_server_poll(hoszp_server* s, hoszp_completion* out, uint32_t max, uint32_t* count,
                      uint64_t wait_us) {
  if (!s || !count || (max && !out)) return HOSZP_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_us)
    s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [s]() { return !s->done.empty(); });
  uint32_t n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  *count = n;
  return HOSZP_OK;
}

int hoszp_server_release(hoszp_server* s, void* d_out) {
  if (!s || !d_out) return HOSZP_ERR_ARG;
  const uint8_t* p = static_cast<const uint8_t*>(d_out);
  const uint8_t* b = static_cast<const uint8_t*>(s->arena_mem);
  if (p < b || p >= b + s->arena.size()) return HOSZP_ERR_ARG;
  bool ok;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    ok = s->arena.release((uint64_t)(p - b));
  }
  s->cv_work.notify_all();
  return ok ? HOSZP_OK : HOSZP_ERR_ARG;
}

uint64_t hoszp_server_now_us(const hoszp_server* s) { return s ? s->now() : 0; }

int hoszp_server_get_stats(hoszp_server* s, hoszp_server_stats* st) {
  if (!s || !st) return HOSZP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->pending = s->pending.size();
  st->in_flight = s->in_flight;
  st->arena_bytes = s->arena.size();
  st->arena_in_use = s->arena.in_use();
  st->arena_peak = s->arena.peak();
  st->workspace_bytes = s->workspace_bytes;
  st->max_in_flight = s->max_in_flight;
  return HOSZP_OK;
}

}  // extern "C"
