// Serving loop around the fused path: requests with host-memory buffers
// arrive at any time; a dispatcher thread admits them in arrival order (a
// free lane and room in the device-memory budget), copies their inputs into
// the lane's device arena, replays the lane's CUDA graph for the request's
// shape bucket and copies the image back, all on the lane's stream, so lanes
// overlap copies of one request with the kernels of another.  A completion
// thread polls the lanes' events and records each request's latency (submit
// to result in host memory).  The paper times single frames only (Sec. 5);
// this is the deployment layer.
//
// Each lane owns a private latent: a request's scene latent (resident, LRU)
// is copied into it on the lane's stream before the graph runs, so a graph
// captured once per (lane, bucket) never needs rebinding.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Bucket {
  int h, w, K;
  bool operator<(const Bucket& o) const { return std::tie(h, w, K) < std::tie(o.h, o.w, o.K); }
};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of one request's buffers in a lane arena.
struct ArenaMap {
  size_t gbuf, tbuf, counts, out, end;
  ArenaMap(int K, int h, int w) {
    const size_t P = static_cast<size_t>(h) * w;
    gbuf = 0;
    tbuf = up256(P * gn::kGC * 4);
    counts = tbuf + up256(P * gn::kTC * 4 * static_cast<size_t>(K));
    out = counts + up256(P);
    end = out + up256(P * gn::kOut * 4);
  }
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  // timing marks of the request in flight: work started, inputs on the
  // device, image rendered (`done`: image in host memory)
  cudaEvent_t t_start = nullptr, t_in = nullptr, t_kern = nullptr;
  uint8_t* arena = nullptr;
  gn_latent latent;  // lane-private latent (device)
  std::map<Bucket, gn_graph*> graphs;
  bool busy = false;    // holds a job (set by the dispatcher before it enqueues the job's work)
  bool issued = false;  // the job's work and its `done` event are enqueued: only then is the
                        // event the job's own (before, it still holds the previous job's)
  uint64_t ticket = 0;
};

struct Job {
  gn_request req;
  Clock::time_point t_submit, t_dispatch, t_issued;  // submitted, taken by the dispatcher, enqueued
  size_t bytes = 0;
  int scene_slot = -1;
  bool done = false;
  int status = GN_OK;
  double latency_ms = 0.0;
  gn_request_times times = {};
};

// A scene slot is empty (id < 0, not encoding), resident (id >= 0) or being
// (re-)encoded by one glassnet_server_add_scene call (encoding: no other call
// may take it, and no request can name it).
struct Scene {
  int id = -1;
  bool encoding = false;
  gn_latent* latent = nullptr;
  uint64_t last_use = 0;
  int in_flight = 0;
};

int err(int code, const char* fmt, const char* a = "", const char* b = "") {
  char buf[320];
  std::snprintf(buf, sizeof(buf), fmt, a, b);
  return gn::set_error(code, buf);
}

}  // namespace

struct gn_server {
  gn_model* model = nullptr;
  gn_server_config cfg{};
  size_t latent_bytes = 0;
  std::vector<Lane> lanes;
  std::vector<Scene> scenes;
  int next_scene_id = 0;
  uint64_t use_clock = 0;

  std::mutex mu;
  std::condition_variable cv;  // any state change
  std::deque<uint64_t> queue;
  std::map<uint64_t, Job> jobs;
  uint64_t next_ticket = 1;
  size_t bytes_in_flight = 0;
  std::vector<double> latencies;
  uint64_t submitted = 0, completed = 0;
  double pixels_done = 0.0;
  bool stop = false;
  bool preparing = false;  // glassnet_server_prepare is capturing graphs: no dispatch
  std::thread dispatcher, completer;

  void dispatch_loop();
  void complete_loop();
  int issue(Lane& lane, Job& job);
};

// The lane's graph of a shape bucket, captured on first use.
int gn_server_bucket_graph(gn_model* model, Lane& lane, const Bucket& bk,
                           std::map<Bucket, gn_graph*>::iterator* out) {
  auto it = lane.graphs.find(bk);
  if (it == lane.graphs.end()) {
    const ArenaMap am(bk.K, bk.h, bk.w);
    gn_frame f;
    f.latent = &lane.latent;
    f.gbuf = reinterpret_cast<const float*>(lane.arena + am.gbuf);
    f.tbuf = bk.K > 0 ? reinterpret_cast<const float*>(lane.arena + am.tbuf) : nullptr;
    f.layer_count = lane.arena + am.counts;
    f.K = bk.K;
    f.h = bk.h;
    f.w = bk.w;
    f.out = reinterpret_cast<float*>(lane.arena + am.out);
    gn_graph* g = nullptr;
    const int rc = glassnet_graph_create(model, &f, 1, &g);
    if (rc != GN_OK) return rc;
    it = lane.graphs.emplace(bk, g).first;
  }
  *out = it;
  return GN_OK;
}

int gn_server::issue(Lane& lane, Job& job) {
  const gn_request& r = job.req;
  const Bucket bk{r.h, r.w, r.K};
  const ArenaMap am(r.K, r.h, r.w);
  std::map<Bucket, gn_graph*>::iterator it;
  const int grc = gn_server_bucket_graph(model, lane, bk, &it);
  if (grc != GN_OK) return grc;
  const size_t P = static_cast<size_t>(r.h) * r.w;
  cudaError_t e = cudaEventRecord(lane.t_start, lane.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lane.latent.d, scenes[job.scene_slot].latent->d, latent_bytes,
                        cudaMemcpyDeviceToDevice, lane.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lane.arena + am.gbuf, r.gbuf, P * gn::kGC * 4, cudaMemcpyHostToDevice,
                        lane.stream);
  if (e == cudaSuccess && r.K > 0)
    e = cudaMemcpyAsync(lane.arena + am.tbuf, r.tbuf, P * gn::kTC * 4 * static_cast<size_t>(r.K),
                        cudaMemcpyHostToDevice, lane.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lane.arena + am.counts, r.layer_count, P, cudaMemcpyHostToDevice,
                        lane.stream);
  if (e == cudaSuccess) e = cudaEventRecord(lane.t_in, lane.stream);
  if (e != cudaSuccess) return err(GN_ECUDA, "request copies: %s", cudaGetErrorString(e));
  int rc = glassnet_graph_launch(it->second, lane.stream);
  if (rc != GN_OK) return rc;
  e = cudaEventRecord(lane.t_kern, lane.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r.out, lane.arena + am.out, P * gn::kOut * 4, cudaMemcpyDeviceToHost,
                        lane.stream);
  if (e == cudaSuccess) e = cudaEventRecord(lane.done, lane.stream);
  if (e != cudaSuccess) return err(GN_ECUDA, "result copy: %s", cudaGetErrorString(e));
  return GN_OK;
}

void gn_server::dispatch_loop() {
  cudaSetDevice(model->device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    int free_lane = -1;
    cv.wait(lk, [&] {
      if (stop) return true;
      if (queue.empty() || preparing) return false;
      const Job& j = jobs[queue.front()];
      if (bytes_in_flight + j.bytes > cfg.budget_bytes) return false;
      for (size_t i = 0; i < lanes.size(); ++i)
        if (!lanes[i].busy) {
          free_lane = static_cast<int>(i);
          return true;
        }
      return false;
    });
    if (stop) break;
    const uint64_t t = queue.front();
    queue.pop_front();
    Job& job = jobs[t];
    job.t_dispatch = Clock::now();
    Lane& lane = lanes[free_lane];
    lane.busy = true;
    lane.ticket = t;
    bytes_in_flight += job.bytes;
    lk.unlock();
    const int rc = issue(lane, job);
    lk.lock();
    if (rc != GN_OK) {  // nothing is in flight for this lane: fail the request now
      job.status = rc;
      job.done = true;
      lane.busy = false;
      bytes_in_flight -= job.bytes;
      scenes[job.scene_slot].in_flight--;
    } else {
      job.t_issued = Clock::now();
      lane.issued = true;  // the completer may query the lane's event from now on
    }
    cv.notify_all();
  }
}

void gn_server::complete_loop() {
  cudaSetDevice(model->device);
  while (true) {
    std::vector<int> busy;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] {
        if (stop) return true;
        for (const Lane& l : lanes)
          if (l.busy && l.issued) return true;
        return false;
      });
      if (stop) return;
      for (size_t i = 0; i < lanes.size(); ++i)
        if (lanes[i].busy && lanes[i].issued) busy.push_back(static_cast<int>(i));
    }
    bool any = false;
    for (int i : busy) {
      const cudaError_t q = cudaEventQuery(lanes[i].done);
      if (q == cudaErrorNotReady) continue;
      any = true;
      const auto now = Clock::now();
      std::lock_guard<std::mutex> lk(mu);
      Lane& lane = lanes[i];
      Job& job = jobs[lane.ticket];
      job.status = q == cudaSuccess ? GN_OK : GN_ECUDA;
      auto ms = [](Clock::time_point a, Clock::time_point b) {
        return std::chrono::duration<double, std::milli>(b - a).count();
      };
      job.latency_ms = ms(job.t_submit, now);
      job.times.queue_ms = ms(job.t_submit, job.t_dispatch);
      job.times.enqueue_ms = ms(job.t_dispatch, job.t_issued);
      job.times.device_ms = ms(job.t_issued, now);
      job.times.total_ms = job.latency_ms;
      float a = 0.0f, b = 0.0f, c = 0.0f;  // device timeline of the lane's stream
      if (q == cudaSuccess && cudaEventElapsedTime(&a, lane.t_start, lane.t_in) == cudaSuccess &&
          cudaEventElapsedTime(&b, lane.t_in, lane.t_kern) == cudaSuccess &&
          cudaEventElapsedTime(&c, lane.t_kern, lane.done) == cudaSuccess) {
        job.times.copy_in_ms = a;
        job.times.render_ms = b;
        job.times.copy_out_ms = c;
      }
      job.done = true;
      latencies.push_back(job.latency_ms);
      ++completed;
      pixels_done += static_cast<double>(job.req.h) * job.req.w;
      bytes_in_flight -= job.bytes;
      scenes[job.scene_slot].in_flight--;
      lane.busy = false;
      lane.issued = false;
      cv.notify_all();
    }
    if (!any) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

extern "C" {

int glassnet_server_create(gn_model* m, const gn_server_config* cfg, gn_server** out) {
  if (!m || !cfg || !out) return gn::set_error(GN_EINVAL, "model, config and out must be non-NULL");
  *out = nullptr;
  if (m->precision == GN_FP32_PLAIN)
    return gn::set_error(GN_EUNSUPPORTED, "the server runs a fused precision");
  if (m->precision == GN_FP8_FUSED && !m->fp8_ready)
    return gn::set_error(GN_EINVAL, "FP8 model is not calibrated (glassnet_calibrate_fp8)");
  if (cfg->n_streams < 1 || cfg->n_streams > 16 || cfg->max_scenes < 1 || cfg->max_h < 1 ||
      cfg->max_w < 1 || cfg->max_K < 0 || cfg->max_K > gn::kMaxK)
    return gn::set_error(GN_EINVAL, "config outside n_streams 1..16, max_scenes >= 1, max sizes >= 1");
  gn_server* s = new (std::nothrow) gn_server();
  if (!s) return gn::set_error(GN_ENOMEM, "host allocation failed");
  s->model = m;
  s->cfg = *cfg;
  s->latent_bytes = (static_cast<size_t>(m->Z) + 2 * m->H + gn::kScene) * sizeof(float);
  const size_t arena = ArenaMap(cfg->max_K, cfg->max_h, cfg->max_w).end;
  s->lanes.resize(cfg->n_streams);
  cudaSetDevice(m->device);
  for (Lane& l : s->lanes) {
    l.latent.H = m->H;
    l.latent.Z = m->Z;
    if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&l.done) != cudaSuccess || cudaEventCreate(&l.t_start) != cudaSuccess ||
        cudaEventCreate(&l.t_in) != cudaSuccess || cudaEventCreate(&l.t_kern) != cudaSuccess ||
        cudaMalloc(&l.arena, arena) != cudaSuccess ||
        cudaMalloc(&l.latent.d, s->latent_bytes) != cudaSuccess) {
      glassnet_server_destroy(s);
      return gn::set_error(GN_ENOMEM, "lane allocation failed");
    }
  }
  s->scenes.resize(cfg->max_scenes);
  s->dispatcher = std::thread([s] { s->dispatch_loop(); });
  s->completer = std::thread([s] { s->complete_loop(); });
  *out = s;
  return GN_OK;
}

int glassnet_server_add_scene(gn_server* s, const float* scene, int* scene_id) {
  if (!s || !scene || !scene_id) return gn::set_error(GN_EINVAL, "server, scene and id must be non-NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  // an empty slot, else the least recently used resident one once no request
  // uses it; slots that another call is encoding are never taken
  int slot = -1;
  s->cv.wait(lk, [&] {
    slot = -1;
    for (size_t i = 0; i < s->scenes.size(); ++i)
      if (s->scenes[i].id < 0 && !s->scenes[i].encoding) {
        slot = static_cast<int>(i);
        return true;
      }
    for (size_t i = 0; i < s->scenes.size(); ++i) {
      const Scene& c = s->scenes[i];
      if (c.encoding || c.in_flight > 0) continue;
      if (slot < 0 || c.last_use < s->scenes[slot].last_use) slot = static_cast<int>(i);
    }
    return slot >= 0;
  });
  Scene& sc = s->scenes[slot];
  sc.id = -1;  // not usable while it is being re-encoded
  sc.encoding = true;
  gn_latent* old = sc.latent;
  sc.latent = nullptr;
  lk.unlock();
  if (old) glassnet_free_latent(old);
  // encode on a private stream, so that adding a scene does not wait for the
  // lanes' requests in flight
  gn_latent* lat = nullptr;
  cudaStream_t st = nullptr;
  cudaSetDevice(s->model->device);
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  int rc = e == cudaSuccess ? glassnet_encode_scene(s->model, scene, &lat, st)
                            : err(GN_ECUDA, "scene stream: %s", cudaGetErrorString(e));
  if (rc == GN_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      glassnet_free_latent(lat);
      lat = nullptr;
      rc = err(GN_ECUDA, "scene encoder failed: %s", cudaGetErrorString(e));
    }
  }
  if (st) cudaStreamDestroy(st);
  lk.lock();
  sc.encoding = false;
  if (rc != GN_OK) {  // the slot is empty again
    s->cv.notify_all();
    return rc;
  }
  sc.latent = lat;
  sc.id = s->next_scene_id++;
  sc.last_use = ++s->use_clock;
  *scene_id = sc.id;
  s->cv.notify_all();
  return GN_OK;
}

int glassnet_server_prepare(gn_server* s, int h, int w, int K) {
  if (!s) return gn::set_error(GN_EINVAL, "server is NULL");
  if (K < 0 || K > s->cfg.max_K || h < 1 || w < 1 || h > s->cfg.max_h || w > s->cfg.max_w)
    return gn::set_error(GN_EINVAL, "bucket outside the server's maximum");
  {
    // the lanes must be idle; the dispatcher admits nothing while their
    // graphs are captured (a lane's `busy` means a request in flight, which
    // the completion thread would look for)
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->preparing) return gn::set_error(GN_EINVAL, "another prepare is running");
    if (!s->queue.empty()) return gn::set_error(GN_EINVAL, "requests are queued");
    for (const Lane& l : s->lanes)
      if (l.busy) return gn::set_error(GN_EINVAL, "requests are in flight");
    s->preparing = true;
  }
  cudaSetDevice(s->model->device);
  int rc = GN_OK;
  for (Lane& l : s->lanes) {
    std::map<Bucket, gn_graph*>::iterator it;
    if ((rc = gn_server_bucket_graph(s->model, l, Bucket{h, w, K}, &it)) != GN_OK) break;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->preparing = false;
  s->cv.notify_all();
  return rc;
}

int glassnet_server_submit(gn_server* s, const gn_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return gn::set_error(GN_EINVAL, "server, request and ticket must be non-NULL");
  const gn_request& r = *req;
  if (r.K < 0 || r.K > s->cfg.max_K || r.h < 1 || r.w < 1 || r.h > s->cfg.max_h ||
      r.w > s->cfg.max_w || static_cast<long long>(r.h) * r.w > static_cast<long long>(s->cfg.max_h) * s->cfg.max_w)
    return gn::set_error(GN_EINVAL, "request size outside the server's maximum");
  if (!r.gbuf || !r.layer_count || !r.out || (r.K > 0 && !r.tbuf))
    return gn::set_error(GN_EINVAL, "request buffers must be non-NULL");
  const size_t bytes = ArenaMap(r.K, r.h, r.w).end;
  if (bytes > s->cfg.budget_bytes)
    return gn::set_error(GN_EINVAL, "request larger than the device-memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  int slot = -1;
  for (size_t i = 0; i < s->scenes.size(); ++i)
    if (s->scenes[i].id == r.scene && r.scene >= 0) slot = static_cast<int>(i);
  if (slot < 0) return gn::set_error(GN_EINVAL, "scene id is not resident");
  s->scenes[slot].in_flight++;
  s->scenes[slot].last_use = ++s->use_clock;
  const uint64_t t = s->next_ticket++;
  Job& j = s->jobs[t];
  j.req = r;
  j.t_submit = Clock::now();
  j.bytes = bytes;
  j.scene_slot = slot;
  s->queue.push_back(t);
  ++s->submitted;
  *ticket = t;
  s->cv.notify_all();
  return GN_OK;
}

int glassnet_server_wait_times(gn_server* s, uint64_t ticket, gn_request_times* times) {
  if (!s) return gn::set_error(GN_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return gn::set_error(GN_EINVAL, "unknown ticket");
  s->cv.wait(lk, [&] { return it->second.done || s->stop; });
  if (!it->second.done) return gn::set_error(GN_EINVAL, "server stopped");
  const int rc = it->second.status;
  if (times) *times = it->second.times;
  s->jobs.erase(it);
  if (rc != GN_OK) return gn::set_error(rc, "request failed on the device");
  return GN_OK;
}

int glassnet_server_wait(gn_server* s, uint64_t ticket, double* latency_ms) {
  gn_request_times t;
  const int rc = glassnet_server_wait_times(s, ticket, &t);
  if (rc == GN_OK && latency_ms) *latency_ms = t.total_ms;
  return rc;
}

int glassnet_server_stats(gn_server* s, gn_server_stats* out) {
  if (!s || !out) return gn::set_error(GN_EINVAL, "server and stats must be non-NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->latencies;
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->pixels = s->pixels_done;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {  // nearest rank
      size_t k = static_cast<size_t>(p / 100.0 * static_cast<double>(v.size()) + 0.999999);
      k = std::min(std::max<size_t>(k, 1), v.size());
      return v[k - 1];
    };
    out->p50_ms = pct(50.0);
    out->p99_ms = pct(99.0);
    out->max_ms = v.back();
    double sum = 0.0;
    for (double x : v) sum += x;
    out->mean_ms = sum / static_cast<double>(v.size());
  }
  return GN_OK;
}

void glassnet_server_destroy(gn_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // let admitted and queued requests finish first
    s->cv.wait(lk, [&] {
      if (!s->queue.empty()) return false;
      for (const Lane& l : s->lanes)
        if (l.busy) return false;
      return true;
    });
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->dispatcher.joinable()) s->dispatcher.join();
  if (s->completer.joinable()) s->completer.join();
  for (Lane& l : s->lanes) {
    if (l.stream) cudaStreamSynchronize(l.stream);
    for (auto& kv : l.graphs) glassnet_graph_free(kv.second);
    if (l.arena) cudaFree(l.arena);
    if (l.latent.d) cudaFree(l.latent.d);
    if (l.done) cudaEventDestroy(l.done);
    if (l.t_start) cudaEventDestroy(l.t_start);
    if (l.t_in) cudaEventDestroy(l.t_in);
    if (l.t_kern) cudaEventDestroy(l.t_kern);
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  for (Scene& sc : s->scenes)
    if (sc.latent) glassnet_free_latent(sc.latent);
  delete s;
}

}  // extern "C"
