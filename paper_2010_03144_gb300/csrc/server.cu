// Request server: compress / decompress / verify requests admitted continuously.
//
// One scheduler thread owns `slots` CUDA streams. A request is admitted as soon as a slot is
// free and the device memory it needs (workspace, plus the output when the server provides
// it) fits in the remaining HBM budget; admitted requests run concurrently on their streams,
// and each slot is handed to the next pending request (first come, first served) the moment
// its completion event fires, so requests that arrive while others run join the device work
// without waiting for a batch boundary. Memory comes from a private stream-ordered pool. The
// compressed streams (with their code tables and sum_dc checksums) and any server-provided
// outputs stay in device memory until the client releases them. Nothing here changes the
// arithmetic: every request runs the same kernels as the single-field entry points.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.h"

namespace sdcsz {
namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Req {
  sdcsz_request r;
  double t_submit = 0.0, t_admit = 0.0;
  Geo g;
  Hdr h;
  bool parsed = false;
  size_t ws_bytes = 0, out_bytes = 0;
  void* ws = nullptr;
  void* out = nullptr;  // server-provided output (or null)
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  State* h_state = nullptr;  // pinned copy of the request's State
  bool busy = false;
  Req q;
};

}  // namespace
}  // namespace sdcsz

struct sdcsz_server {
  sdcsz_server_config cfg;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  cudaMemPool_t pool = nullptr;
  cudaStream_t aux = nullptr;  // header reads and releases
  uint8_t* h_hdr = nullptr;
  std::vector<sdcsz::Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<sdcsz::Req> pending;
  std::deque<sdcsz_completion> completed;
  std::unordered_map<uint64_t, std::pair<void*, size_t>> held;  // outputs kept for the client
  uint64_t used = 0, peak = 0, admitted = 0, finished = 0;
  bool stop = false;
  std::thread th;
};

namespace sdcsz {
namespace {

// Budget bytes a request needs while it runs, and how much of it stays held afterwards.
int request_need(sdcsz_server* S, Req& q) {
  const sdcsz_request& r = q.r;
  if (r.op == SDCSZ_OP_COMPRESS) {
    int rc = make_geo(&r.params, &q.g);
    if (rc) return rc;
    q.ws_bytes = plan_ws(q.g).total;
    size_t cap = 0;
    if ((rc = sdcsz_compress_bound(&r.params, &cap))) return rc;
    q.out_bytes = r.d_out ? 0 : align256(cap);
    if (r.d_out && r.out_cap < cap) return SDCSZ_ECAPACITY;
    return SDCSZ_OK;
  }
  if (r.op != SDCSZ_OP_DECOMPRESS && r.op != SDCSZ_OP_VERIFY) return SDCSZ_EINVAL;
  if (!q.parsed) {
    if (!r.d_in || r.in_bytes < (size_t)kHeaderBytes) return SDCSZ_EFORMAT;
    if (cudaMemcpyAsync(S->h_hdr, r.d_in, kHeaderBytes, cudaMemcpyDeviceToHost, S->aux) != cudaSuccess ||
        cudaStreamSynchronize(S->aux) != cudaSuccess)
      return SDCSZ_ECUDA;
    const int rc = parse_header(S->h_hdr, r.in_bytes, &q.h, nullptr);
    if (rc) return rc;
    q.parsed = true;
  }
  const uint64_t field = q.h.g.N * (q.h.g.dtype ? 8 : 4);
  q.ws_bytes = decode_ws_bytes(q.h) + (r.op == SDCSZ_OP_VERIFY ? align256(q.h.g.nb) : 0);
  q.out_bytes = (r.op == SDCSZ_OP_DECOMPRESS && !r.d_out) ? align256(field) : 0;
  if (r.op == SDCSZ_OP_DECOMPRESS && r.d_out && r.out_cap < field) return SDCSZ_ECAPACITY;
  return SDCSZ_OK;
}

void finish(sdcsz_server* S, Req& q, int status, const State* st) {
  sdcsz_completion c;
  std::memset(&c, 0, sizeof(c));
  c.id = q.r.id;
  c.op = q.r.op;
  c.status = status;
  c.t_submit = q.t_submit;
  c.t_admit = q.t_admit;
  c.t_done = now_s(S->t0);
  if (st) {
    if (q.r.op == SDCSZ_OP_COMPRESS) {
      fill_report(*st, q.g.nb, &c.report);
      c.d_result = q.r.d_out ? q.r.d_out : q.out;
      c.result_bytes = status ? 0 : (size_t)st->total_bytes;
    } else {
      State hs = *st;
      hs.n_reg = q.h.n_reg;
      hs.n_unpred = q.h.n_unpred;
      hs.total_bytes = q.h.total;
      hs.eb = q.h.eb;
      fill_report(hs, q.h.g.nb, &c.report);
      if (q.r.op == SDCSZ_OP_DECOMPRESS) {
        c.d_result = q.r.d_out ? q.r.d_out : q.out;
        c.result_bytes = status ? 0 : (size_t)(q.h.g.N * (q.h.g.dtype ? 8 : 4));
      }
    }
  }
  if (q.out) {
    if (status == SDCSZ_OK || status == SDCSZ_ESDC) {
      S->held[q.r.id] = {q.out, q.out_bytes};  // until sdcsz_server_release
    } else {
      cudaFreeAsync(q.out, S->aux);
      S->used -= q.out_bytes;
      c.d_result = nullptr;
    }
  }
  S->completed.push_back(c);
  ++S->finished;
}

// Enqueue an admitted request on its slot (called without the lock).
int launch(sdcsz_server* S, Slot& sl) {
  Req& q = sl.q;
  const sdcsz_request& r = q.r;
  cudaStream_t s = sl.s;
  if (cudaMallocFromPoolAsync(&q.ws, q.ws_bytes, S->pool, s) != cudaSuccess) return SDCSZ_ECUDA;
  if (q.out_bytes && cudaMallocFromPoolAsync(&q.out, q.out_bytes, S->pool, s) != cudaSuccess) return SDCSZ_ECUDA;
  int rc;
  State* st;
  if (r.op == SDCSZ_OP_COMPRESS) {
    void* out = r.d_out ? r.d_out : q.out;
    const size_t cap = r.d_out ? r.out_cap : q.out_bytes;
    rc = compress_impl(r.d_in, &r.params, out, cap, nullptr, q.ws, q.ws_bytes, nullptr, s, r.d_flips, r.n_flips);
    st = static_cast<State*>(q.ws);
  } else {
    st = static_cast<State*>(q.ws);
    const bool write = r.op == SDCSZ_OP_DECOMPRESS;
    void* field = write ? (r.d_out ? r.d_out : q.out) : nullptr;
    const size_t fb = write ? (r.d_out ? r.out_cap : q.out_bytes) : 0;
    uint8_t* base = static_cast<uint8_t*>(q.ws);
    uint8_t* raw = base + align256(sizeof(State));  // the lossless stage's scratch, when there is one
    uint8_t* status = write ? nullptr : base + decode_ws_bytes(q.h);
    uint8_t* wave = wave_decode_ws_bytes(q.h.g) ? base + decode_ws_min(q.h) : nullptr;  // the two-pass decoder's
    rc = decode_enqueue(r.d_in, r.in_bytes, q.h, field, fb, status, write ? nullptr : r.d_original, write, st, s,
                        r.d_flips, r.n_flips, raw, wave);
  }
  if (rc) return rc;
  if (cudaMemcpyAsync(sl.h_state, st, sizeof(State), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaEventRecord(sl.done, s) != cudaSuccess) return SDCSZ_ECUDA;
  return SDCSZ_OK;
}

void release_ws(sdcsz_server* S, Slot& sl) {
  if (sl.q.ws) cudaFreeAsync(sl.q.ws, sl.s);
  sl.q.ws = nullptr;
  S->used -= sl.q.ws_bytes;
}

void scheduler(sdcsz_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progressed = false, any_busy = false;
    // retire finished requests: their slots and workspaces go back at once
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      int status = e == cudaSuccess ? map_error(sl.h_state->error) : SDCSZ_ECUDA;
      if (!status && sl.q.r.op != SDCSZ_OP_COMPRESS && sl.h_state->uncorrectable) status = SDCSZ_ESDC;
      if (e != cudaSuccess) cudaGetLastError();
      release_ws(S, sl);
      finish(S, sl.q, status, e == cudaSuccess ? sl.h_state : nullptr);
      sl.busy = false;
      progressed = true;
    }
    // admit pending requests in arrival order while a slot and the budget allow
    for (auto& sl : S->slots) {
      if (sl.busy || S->pending.empty()) continue;
      Req& q = S->pending.front();
      const int rc = request_need(S, q);
      if (rc || q.ws_bytes + q.out_bytes > S->cfg.hbm_budget) {
        finish(S, q, rc ? rc : SDCSZ_ECAPACITY, nullptr);
        S->pending.pop_front();
        progressed = true;
        continue;
      }
      if (S->used + q.ws_bytes + q.out_bytes > S->cfg.hbm_budget) break;  // wait for memory
      sl.q = q;
      S->pending.pop_front();
      S->used += sl.q.ws_bytes + sl.q.out_bytes;
      S->peak = std::max(S->peak, S->used);
      sl.q.t_admit = now_s(S->t0);
      sl.busy = true;
      ++S->admitted;
      lk.unlock();
      const int lr = launch(S, sl);
      lk.lock();
      if (lr) {
        cudaGetLastError();
        cudaStreamSynchronize(sl.s);
        release_ws(S, sl);
        finish(S, sl.q, lr, nullptr);
        sl.busy = false;
      } else {
        any_busy = true;
      }
      progressed = true;
    }
    if (progressed) S->cv_done.notify_all();
    if (S->stop && S->pending.empty() && !any_busy) break;
    if (!progressed) {
      if (any_busy) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      } else {
        S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      }
    }
  }
}

}  // namespace
}  // namespace sdcsz

using namespace sdcsz;

extern "C" {

int sdcsz_server_create(const sdcsz_server_config* cfg, sdcsz_server** out) {
  if (!cfg || !out || cfg->slots == 0 || cfg->slots > 64 || cfg->hbm_budget == 0) return SDCSZ_EINVAL;
  *out = nullptr;
  sdcsz_server* S = new sdcsz_server();
  S->cfg = *cfg;
  S->t0 = std::chrono::steady_clock::now();
  int rc = SDCSZ_OK;
  if (cudaGetDevice(&S->device) != cudaSuccess) rc = SDCSZ_ECUDA;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->device;
  if (!rc && cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) rc = SDCSZ_ECUDA;
  if (!rc) {
    uint64_t keep = cfg->hbm_budget;  // keep freed memory cached up to the budget
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (!rc && cudaStreamCreateWithFlags(&S->aux, cudaStreamNonBlocking) != cudaSuccess) rc = SDCSZ_ECUDA;
  if (!rc && cudaMallocHost(&S->h_hdr, kHeaderBytes) != cudaSuccess) rc = SDCSZ_ECUDA;
  S->slots.resize(cfg->slots);
  for (auto& sl : S->slots) {
    if (rc) break;
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&sl.h_state, sizeof(State)) != cudaSuccess)
      rc = SDCSZ_ECUDA;
  }
  if (rc) {
    sdcsz_server_destroy(S);
    return rc;
  }
  S->th = std::thread(scheduler, S);
  *out = S;
  return SDCSZ_OK;
}

int sdcsz_server_submit(sdcsz_server* S, const sdcsz_request* r) {
  if (!S || !r || !r->d_in) return SDCSZ_EINVAL;
  if (r->n_flips && !r->d_flips) return SDCSZ_EINVAL;
  Req q;
  q.r = *r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return SDCSZ_EINVAL;
    q.t_submit = now_s(S->t0);
    S->pending.push_back(q);
  }
  S->cv_work.notify_one();
  return SDCSZ_OK;
}

int sdcsz_server_poll(sdcsz_server* S, sdcsz_completion* out, uint32_t max, uint32_t* n, uint32_t wait_us) {
  if (!S || !n || (max && !out)) return SDCSZ_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->completed.empty() && wait_us)
    S->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !S->completed.empty(); });
  uint32_t k = 0;
  while (k < max && !S->completed.empty()) {
    out[k++] = S->completed.front();
    S->completed.pop_front();
  }
  *n = k;
  return SDCSZ_OK;
}

int sdcsz_server_release(sdcsz_server* S, uint64_t id) {
  if (!S) return SDCSZ_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->held.find(id);
  if (it == S->held.end()) return SDCSZ_EINVAL;
  cudaFreeAsync(it->second.first, S->aux);
  S->used -= it->second.second;
  S->held.erase(it);
  S->cv_work.notify_one();
  return SDCSZ_OK;
}

int sdcsz_server_get_stats(sdcsz_server* S, sdcsz_server_stats* out) {
  if (!S || !out) return SDCSZ_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  out->pending = S->pending.size();
  uint64_t busy = 0;
  for (auto& sl : S->slots) busy += sl.busy;
  out->in_flight = busy;
  out->admitted = S->admitted;
  out->completed = S->finished;
  out->bytes_in_use = S->used;
  out->peak_bytes = S->peak;
  return SDCSZ_OK;
}

void sdcsz_server_destroy(sdcsz_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  for (auto& kv : S->held) cudaFreeAsync(kv.second.first, S->aux);
  if (S->aux) cudaStreamSynchronize(S->aux);
  for (auto& sl : S->slots) {
    if (sl.s) cudaStreamSynchronize(sl.s);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.s) cudaStreamDestroy(sl.s);
    if (sl.h_state) cudaFreeHost(sl.h_state);
  }
  if (S->aux) cudaStreamDestroy(S->aux);
  if (S->h_hdr) cudaFreeHost(S->h_hdr);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
}

}  // extern "C"
