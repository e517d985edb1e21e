// serve.cpp -- continuous-batching render server over one resident scene.
//
// A scheduler thread forms batches whenever a stream is idle.  A batch takes
// the oldest queued request and then, in arrival order, further queued
// requests of the same kernel class (coherent cameras and explicit rays;
// divergent cameras -- fisheye, panorama; span-parallel rays -- spinning
// LiDARs), up to SALF_MAX_BATCH, as long as their outputs fit in a fixed
// device arena (admission by memory).  Each class has its own kernel shape,
// so a batch is one launch of the forward kernel (each request keeps its own
// sensor, options and output slice) and batches of different classes run
// side by side on different streams.  Requests that arrive while batches run
// join the next batch as soon as a stream frees up, so work from different
// requests overlaps on the device.  Completion is signalled by a host
// function queued behind each batch on its stream.  Rays are independent and
// the batched launch runs the same per-ray code as salf_render_rays, so a
// request's outputs do not depend on what it was batched with.
//
// Host-side fault injection for tests (environment variable SALF_SERVE_FAULT):
//   "launch_fail:N"  the N-th batch (1-based) is not launched and its requests
//                    complete with SALF_ERR_CUDA;
//   "create_oom"     salf_serve_create reports SALF_ERR_OOM.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "salf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum class St { Queued, Running, Done, Failed };

struct Request {
  uint64_t ticket = 0;
  int cls = 0;  // kernel class (batch_class)
  salf_sensor sensor{};
  salf_render_opts opts{};
  ReqDev rd{};
  int64_t rays = 0;
  size_t bytes = 0;
  size_t offset = 0;
  St state = St::Queued;
  salf_status err = SALF_OK;
  float *rgb = nullptr, *depth = nullptr, *opacity = nullptr, *intensity = nullptr;
  uint8_t* valid = nullptr;
  Clock::time_point t_submit, t_done;
};

// First-fit allocator over [0, size) with coalescing free list.
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  size_t used = 0, peak = 0;
  void init(size_t n) {
    size = n;
    free_.clear();
    free_[0] = n;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n;
        const size_t start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used += n;
        peak = std::max(peak, used);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

// Latencies of the most recent completions (a fixed window keeps a long-
// running server's memory and stats cost bounded).
constexpr size_t kLatencyWindow = 1 << 16;

struct salf_server {
  salf_scene* scene = nullptr;
  char* arena_base = nullptr;
  Arena arena;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_busy;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<double> latencies_ms;  // ring of the last kLatencyWindow completions
  size_t lat_next = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool hold = false;
  int64_t submitted = 0, completed = 0, rejected = 0, launches = 0, rays = 0;
  int64_t requests_launched = 0, max_batch = 0, mixed_launches = 0;
  int64_t fail_launch_at = -1;
  std::thread th;
};

namespace {

struct BatchDone {
  salf_server* srv;
  int stream;
  std::vector<uint64_t> tickets;
  salf_status status;
};

void CUDART_CB on_batch_done(void* p) {
  BatchDone* b = static_cast<BatchDone*>(p);
  salf_server* s = b->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const auto now = Clock::now();
    for (uint64_t t : b->tickets) {
      auto it = s->reqs.find(t);
      if (it == s->reqs.end()) continue;
      Request& r = it->second;
      r.state = b->status == SALF_OK ? St::Done : St::Failed;
      r.err = b->status;
      r.t_done = now;
      s->completed++;
      const double ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
      if (s->latencies_ms.size() < kLatencyWindow) {
        s->latencies_ms.push_back(ms);
      } else {
        s->latencies_ms[s->lat_next] = ms;
        s->lat_next = (s->lat_next + 1) % kLatencyWindow;
      }
    }
    s->stream_busy[b->stream]--;
  }
  s->cv_done.notify_all();
  s->cv_sched.notify_all();
  delete b;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Kernel class of a prepared request: requests of one class share a forward
// variant and so a launch (0: pinhole cameras and explicit rays, whole rays;
// 1: fisheye and panorama, whole rays; 2: span-parallel rays).
int batch_class(const ReqDev& d) {
  if (d.seg_shift > 0) return 2;
  return (d.kind == SALF_PINHOLE || d.kind == SALF_RAYS_EXPLICIT) ? 0 : 1;
}

// Output layout of one request inside the arena.
size_t layout(Request& r, char* base) {
  const size_t R = (size_t)r.rays;
  const bool lidar = r.sensor.kind == SALF_LIDAR_SPIN;
  const bool want_int = lidar || r.opts.want_intensity;
  size_t off = 0;
  auto take = [&](size_t n) {
    char* p = base ? base + off : nullptr;
    off += align256(n);
    return p;
  };
  r.rgb = lidar ? nullptr : reinterpret_cast<float*>(take(R * 12));
  r.depth = reinterpret_cast<float*>(take(R * 4));
  r.opacity = reinterpret_cast<float*>(take(R * 4));
  r.intensity = want_int ? reinterpret_cast<float*>(take(R * 4)) : nullptr;
  r.valid = reinterpret_cast<uint8_t*>(take(R));
  return off;
}

void scheduler(salf_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (s->stop && s->pending.empty()) break;
    int idle = -1;
    for (size_t i = 0; i < s->streams.size(); ++i)
      if (s->stream_busy[i] == 0) {
        idle = (int)i;
        break;
      }
    // the oldest request opens a batch; queued requests of its kernel class
    // join it in arrival order while their outputs fit
    std::vector<uint64_t> batch;
    if (idle >= 0 && !s->hold && !s->pending.empty()) {
      const int cls = s->reqs[s->pending.front()].cls;
      for (auto it = s->pending.begin(); it != s->pending.end() && batch.size() < SALF_MAX_BATCH;) {
        Request& r = s->reqs[*it];
        if (r.cls != cls) {
          ++it;
          continue;
        }
        size_t off;
        if (!s->arena.alloc(r.bytes, &off)) break;
        r.offset = off;
        layout(r, s->arena_base + off);
        r.state = St::Running;
        batch.push_back(r.ticket);
        it = s->pending.erase(it);
      }
    }
    if (batch.empty()) {
      s->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    LaunchParams* P = new LaunchParams;
    std::memset(P, 0, sizeof(*P));
    P->S = s->scene->dev;
    int tiles = 0;
    for (uint64_t t : batch) {
      Request& r = s->reqs[t];
      ReqDev& d = P->req[P->n_req++];
      d = r.rd;
      d.rgb = r.rgb;
      d.depth = r.depth;
      d.opacity = r.opacity;
      d.intensity = r.intensity;
      d.valid = r.valid;
      d.want_int = r.intensity != nullptr;
      d.tile_begin = tiles;
      tiles += d.n_tiles;
      s->rays += r.rays;
    }
    P->total_tiles = tiles;
    s->stream_busy[idle]++;
    s->launches++;
    s->requests_launched += (int64_t)batch.size();
    s->max_batch = std::max<int64_t>(s->max_batch, (int64_t)batch.size());
    for (int i = 1; i < P->n_req; ++i)
      if (P->req[i].kind != P->req[0].kind) {
        s->mixed_launches++;
        break;
      }
    const bool inject = s->fail_launch_at > 0 && s->launches == s->fail_launch_at;
    BatchDone* bd = new BatchDone{s, idle, batch, SALF_OK};
    cudaStream_t st = s->streams[idle];
    lk.unlock();
    cudaError_t e = cudaSetDevice(s->scene->device);
    if (inject) {
      bd->status = SALF_ERR_CUDA;
    } else {
      SALF_RANGE("salf_serve_batch");  // one range per batched launch
      if (e == cudaSuccess) e = salf_launch_forward(*P, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        bd->status = SALF_ERR_CUDA;
      }
    }
    delete P;
    e = cudaLaunchHostFunc(st, on_batch_done, bd);
    if (e != cudaSuccess) {
      cudaGetLastError();
      bd->status = SALF_ERR_CUDA;
      on_batch_done(bd);
    }
    lk.lock();
  }
}

}  // namespace

extern "C" salf_status salf_serve_create(salf_scene* scene, size_t budget, int32_t n_streams,
                                         salf_server** out) {
  if (!scene || !out || budget == 0 || n_streams <= 0 || n_streams > 16) {
    salf_set_error("salf_serve_create: bad argument");
    return SALF_ERR_INVALID;
  }
  *out = nullptr;
  const char* f = std::getenv("SALF_SERVE_FAULT");
  std::string fault = f ? f : "";
  if (fault == "create_oom") {
    salf_set_error("salf_serve_create: injected allocation failure");
    return SALF_ERR_OOM;
  }
  cudaError_t e = cudaSetDevice(scene->device);
  if (e != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  salf_server* s = new salf_server();
  s->scene = scene;
  budget = align256(budget);
  e = cudaMalloc(reinterpret_cast<void**>(&s->arena_base), budget);
  if (e != cudaSuccess) {
    delete s;
    return salf_cuda_fail(e, "cudaMalloc(serve arena)");
  }
  s->arena.init(budget);
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      cudaFree(s->arena_base);
      delete s;
      return salf_cuda_fail(e, "cudaStreamCreate");
    }
    s->streams.push_back(st);
    s->stream_busy.push_back(0);
  }
  if (fault.rfind("launch_fail:", 0) == 0) s->fail_launch_at = std::atoll(fault.c_str() + 12);
  s->th = std::thread(scheduler, s);
  *out = s;
  return SALF_OK;
}

extern "C" salf_status salf_serve_submit(salf_server* s, const salf_sensor* sensor,
                                         const salf_render_opts* opts, uint64_t* ticket) {
  if (!s || !sensor || !ticket) {
    salf_set_error("salf_serve_submit: null argument");
    return SALF_ERR_INVALID;
  }
  Request r;
  r.sensor = *sensor;
  if (opts) {
    r.opts = *opts;
  } else {
    std::memset(&r.opts, 0, sizeof(r.opts));
    r.opts.t_min_transmittance = 1e-4f;
  }
  r.opts.visits_cap = 0;
  salf_status st = salf_prepare_request(s->scene, &r.sensor, &r.opts, &r.rd);
  if (st != SALF_OK) return st;
  r.rays = salf_request_rays(&r.sensor);
  r.bytes = layout(r, nullptr);
  r.cls = batch_class(r.rd);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    salf_set_error("salf_serve_submit: server is shutting down");
    return SALF_ERR_SHUTDOWN;
  }
  if (r.bytes > s->arena.size) {
    s->rejected++;
    salf_set_error("salf_serve_submit: request outputs exceed the memory budget");
    return SALF_ERR_INVALID;
  }
  r.ticket = s->next_ticket++;
  r.t_submit = Clock::now();
  *ticket = r.ticket;
  s->pending.push_back(r.ticket);
  s->reqs.emplace(r.ticket, r);
  s->submitted++;
  s->cv_sched.notify_all();
  return SALF_OK;
}

extern "C" salf_status salf_serve_poll(salf_server* s, uint64_t ticket, int32_t timeout_ms,
                                       salf_outputs* result, int32_t* done) {
  if (!s || !done) {
    salf_set_error("salf_serve_poll: null argument");
    return SALF_ERR_INVALID;
  }
  *done = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    salf_set_error("salf_serve_poll: unknown ticket");
    return SALF_ERR_NOT_FOUND;
  }
  auto finished = [&]() {
    auto jt = s->reqs.find(ticket);
    return jt == s->reqs.end() || jt->second.state == St::Done || jt->second.state == St::Failed;
  };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, finished);
  } else if (timeout_ms > 0) {
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
  }
  it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    salf_set_error("salf_serve_poll: ticket released");
    return SALF_ERR_NOT_FOUND;
  }
  Request& r = it->second;
  if (r.state == St::Failed) {
    *done = 1;
    salf_set_error("salf_serve_poll: the request's launch failed");
    return r.err == SALF_OK ? SALF_ERR_CUDA : r.err;
  }
  if (r.state != St::Done) {
    salf_set_error(r.state == St::Queued ? "salf_serve_poll: not admitted yet"
                                         : "salf_serve_poll: still running");
    return SALF_ERR_TIMEOUT;
  }
  *done = 1;
  if (result) {
    std::memset(result, 0, sizeof(*result));
    result->rgb = r.rgb;
    result->depth = r.depth;
    result->opacity = r.opacity;
    result->intensity = r.intensity;
    result->valid = r.valid;
  }
  return SALF_OK;
}

extern "C" salf_status salf_serve_release(salf_server* s, uint64_t ticket) {
  if (!s) {
    salf_set_error("salf_serve_release: null server");
    return SALF_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    salf_set_error("salf_serve_release: unknown ticket");
    return SALF_ERR_NOT_FOUND;
  }
  Request& r = it->second;
  if (r.state == St::Running) {
    salf_set_error("salf_serve_release: request still running");
    return SALF_ERR_AGAIN;
  }
  if (r.state == St::Queued) {
    s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), ticket), s->pending.end());
  } else {
    s->arena.release(r.offset, r.bytes);
  }
  s->reqs.erase(it);
  s->cv_sched.notify_all();
  return SALF_OK;
}

extern "C" salf_status salf_serve_hold(salf_server* s, int32_t hold) {
  if (!s) {
    salf_set_error("salf_serve_hold: null server");
    return SALF_ERR_INVALID;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->hold = hold != 0;
  }
  s->cv_sched.notify_all();
  return SALF_OK;
}

extern "C" salf_status salf_serve_get_stats(salf_server* s, salf_serve_stats* st) {
  if (!s || !st) {
    salf_set_error("salf_serve_get_stats: null argument");
    return SALF_ERR_INVALID;
  }
  std::vector<double> v;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->launches = s->launches;
    st->rays = s->rays;
    st->peak_bytes = (int64_t)s->arena.peak;
    st->requests_launched = s->requests_launched;
    st->max_batch = s->max_batch;
    st->mixed_launches = s->mixed_launches;
    v = s->latencies_ms;  // percentiles are taken outside the lock
  }
  st->latency_window = (int64_t)v.size();
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto q = [&](double p) {
      const size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(p * v.size()) - 1);
      return v[i];
    };
    st->p50_ms = q(0.50);
    st->p99_ms = q(0.99);
    st->max_ms = v.back();
  }
  return SALF_OK;
}

extern "C" void salf_serve_destroy(salf_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->pending.clear();
  }
  s->cv_sched.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->scene->device);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(s->arena_base);
  delete s;
}
