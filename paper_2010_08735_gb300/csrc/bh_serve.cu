// Serving loop: continuous batching of frame requests from many viewers.
//
// Requests queue on the host.  A fixed number of launch slots, each with its
// own stream and staging buffers, take the queued requests in arrival order
// as soon as the slot's previous batch has finished (a CUDA event), so new
// requests join the next launch while earlier ones are still on the GPU and
// launches of different slots overlap on the device.  A batch holds requests
// that share tables, cube map, disc and shading; a request with other
// scene state starts the next batch (this is how a table rebuild is rolled
// out: frames queued against the old tables finish on them).  Admission:
// the frame must fit the memory budget together with every frame queued or
// in flight, and a viewer has at most one frame queued (plus one in flight).
// Viewers on device-resident orbits (bh_serve_submit_orbit) are batched the
// same way; their orbits advance on the device inside the batch, and a
// viewer's request waits on the GPU for the viewer's previous batch when that
// batch is still running on another slot, so each orbit advances in order.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "bh_internal.cuh"

namespace bh {

bh_status render_batch_impl(bh_ctx *ctx, const bh_tables *t, const bh_cubemap *cube, int n,
                            const bh_camera *cams, const bh_disc *disc, const bh_shading *sh,
                            float *const *outs, cudaStream_t s, void *cam_host, void *cam_dev,
                            BatchGraph *bg);
bh_status validate_batch(int n, const bh_camera *cams, const bh_disc *disc, float *const *outs);
bool validate_disc_ext(const bh_disc *d);
size_t cam_const_size();
void serve_destroy(bh_ctx *ctx);
bh_status render_orbit_jobs(bh_ctx *ctx, const bh_tables *t, const bh_cubemap *cube, int n,
                            const OrbitJob *jobs_host, OrbitJob *jobs_dev, void *cams_dev, int *total_dev,
                            const bh_disc *disc, const bh_shading *sh, cudaStream_t s);

using Clock = std::chrono::steady_clock;

struct Request {
  unsigned long long ticket;
  int viewer;
  bool orbit;      // device-resident orbit request (job) rather than a host camera (cam)
  OrbitJob job;
  bh_camera cam;
  bh_disc disc;
  bh_shading sh;
  const bh_tables *tables;
  const bh_cubemap *cube;
  float *out;
  size_t bytes;
  Clock::time_point t_submit;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void *cam_host = nullptr, *cam_dev = nullptr;
  OrbitJob *job_host = nullptr, *job_dev = nullptr;  // orbit batches: pinned staging and device copy
  int *total_dev = nullptr;                          // their tile count, computed on the device
  BatchGraph graph;
  std::vector<Request> batch;
  bool busy = false;
};

constexpr int kSlots = 3;
constexpr int kMaxBatch = 64;

struct ServeState {
  Slot slots[kSlots];
  std::deque<Request> queue;
  std::unordered_map<unsigned long long, double> finished;  // ticket -> latency ms
  std::unordered_map<int, int> queued_per_viewer;
  unsigned long long next_ticket = 1;
  size_t bytes_held = 0;
  std::vector<bh_camera> cams;
  std::vector<float *> outs;
  std::unordered_map<int, int> orbit_slot;  // viewer -> slot running its latest orbit request
};

static bh_status serve_init(bh_ctx *ctx) {
  if (ctx->serve) return BH_OK;
  ServeState *S = new ServeState();
  for (int k = 0; k < kSlots; ++k) {
    Slot &sl = S->slots[k];
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.cam_host, cam_const_size() * kMaxBatch);
    if (e == cudaSuccess) e = cudaMalloc(&sl.cam_dev, cam_const_size() * kMaxBatch);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.job_host, sizeof(OrbitJob) * kMaxBatch);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sl.job_dev, sizeof(OrbitJob) * kMaxBatch + 16);
    if (e == cudaSuccess) sl.total_dev = reinterpret_cast<int *>(sl.job_dev + kMaxBatch);
    if (e != cudaSuccess) {
      ctx->serve = S;
      serve_destroy(ctx);
      return cuda_fail(e, "serve_init");
    }
  }
  ctx->serve = S;
  return BH_OK;
}

void serve_destroy(bh_ctx *ctx) {
  ServeState *S = ctx->serve;
  if (!S) return;
  for (auto &sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    sl.graph.reset();
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.cam_host) cudaFreeHost(sl.cam_host);
    if (sl.cam_dev) cudaFree(sl.cam_dev);
    if (sl.job_host) cudaFreeHost(sl.job_host);
    if (sl.job_dev) cudaFree(sl.job_dev);
  }
  delete S;
  ctx->serve = nullptr;
}

static bool same_disc(const bh_disc &a, const bh_disc &b) {  // field by field: the struct has padding
  return a.r_in == b.r_in && a.r_out == b.r_out && a.t_peak_K == b.t_peak_K && a.density == b.density &&
         a.enabled == b.enabled && a.particles == b.particles && a.time == b.time;
}

static bool same_scene(const Request &a, const Request &b) {
  return a.orbit == b.orbit && a.tables == b.tables && a.cube == b.cube && same_disc(a.disc, b.disc) &&
         a.sh.exposure_disc == b.sh.exposure_disc && a.sh.exposure_stars == b.sh.exposure_stars;
}

// Retire finished slots and start queued requests on free slots.
static bh_status progress(bh_ctx *ctx) {
  TraceRange trace_("bh_serve_progress");
  ServeState *S = ctx->serve;
  for (auto &sl : S->slots) {
    if (!sl.busy) continue;
    cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return cuda_fail(q, "serve: batch");
    Clock::time_point now = Clock::now();
    const int me = (int)(&sl - S->slots);
    for (auto &r : sl.batch) {
      S->finished[r.ticket] = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
      S->bytes_held -= r.bytes;
      if (r.orbit) {
        auto it = S->orbit_slot.find(r.viewer);
        if (it != S->orbit_slot.end() && it->second == me) S->orbit_slot.erase(it);
      }
    }
    sl.batch.clear();
    sl.busy = false;
  }
  for (auto &sl : S->slots) {
    if (sl.busy || S->queue.empty()) continue;
    Request first = S->queue.front();
    S->cams.clear();
    S->outs.clear();
    while (!S->queue.empty() && (int)sl.batch.size() < kMaxBatch && same_scene(S->queue.front(), first)) {
      Request r = S->queue.front();
      S->queue.pop_front();
      if (--S->queued_per_viewer[r.viewer] == 0) S->queued_per_viewer.erase(r.viewer);
      S->cams.push_back(r.cam);
      S->outs.push_back(r.out);
      sl.batch.push_back(r);
    }
    bh_status st;
    if (first.orbit) {
      const int me = (int)(&sl - S->slots);
      for (size_t k = 0; k < sl.batch.size(); ++k) {
        const Request &r = sl.batch[k];
        sl.job_host[k] = r.job;
        auto it = S->orbit_slot.find(r.viewer);
        if (it != S->orbit_slot.end() && it->second != me)
          BH_CUDA(cudaStreamWaitEvent(sl.stream, S->slots[it->second].done, 0));
        S->orbit_slot[r.viewer] = me;
      }
      st = render_orbit_jobs(ctx, first.tables, first.cube, (int)sl.batch.size(), sl.job_host, sl.job_dev,
                             sl.cam_dev, sl.total_dev, &first.disc, &first.sh, sl.stream);
    } else {
      st = render_batch_impl(ctx, first.tables, first.cube, (int)sl.batch.size(), S->cams.data(), &first.disc,
                             &first.sh, S->outs.data(), sl.stream, sl.cam_host, sl.cam_dev, &sl.graph);
    }
    if (st) return st;
    BH_CUDA(cudaEventRecord(sl.done, sl.stream));
    sl.busy = true;
  }
  return BH_OK;
}

}  // namespace bh

using namespace bh;

// Admission and queueing common to both kinds of request (ctx->mu held).
static bh_status enqueue(bh_ctx *ctx, Request &r, const bh_tables *t, const bh_cubemap *cube, int viewer,
                         const bh_disc *disc, const bh_shading *sh, float *out, size_t bytes,
                         unsigned long long *ticket) {
  ServeState *S = ctx->serve;
  if (S->queued_per_viewer.count(viewer)) {
    set_error("bh_serve_submit: viewer %d already has a frame queued", viewer);
    return BH_ERR_BUSY;
  }
  if (ctx->budget && S->bytes_held + bytes > ctx->budget) {
    set_error("bh_serve_submit: frame of %zu bytes exceeds the memory budget", bytes);
    return BH_ERR_BUSY;
  }
  r.ticket = S->next_ticket++;
  r.viewer = viewer;
  r.disc = *disc;
  r.sh = sh ? *sh : bh_shading{1.f, 0.01f};
  r.tables = t;
  r.cube = cube;
  r.out = out;
  r.bytes = bytes;
  r.t_submit = Clock::now();
  S->queue.push_back(r);
  S->queued_per_viewer[viewer]++;
  S->bytes_held += bytes;
  *ticket = r.ticket;
  return progress(ctx);
}

extern "C" bh_status bh_serve_submit(bh_ctx *ctx, const bh_tables *t, const bh_cubemap *cube,
                                     int viewer, const bh_camera *cam, const bh_disc *disc,
                                     const bh_shading *sh, float *out, unsigned long long *ticket) {
  if (!ctx || !t || !cam || !disc || !out || !ticket) {
    set_error("bh_serve_submit: NULL argument");
    return BH_ERR_INVALID_ARG;
  }
  if (viewer < 0 || viewer > 65535) { set_error("bh_serve_submit: viewer out of 0..65535"); return BH_ERR_INVALID_ARG; }
  float *const outs[1] = {out};
  bh_status st = validate_batch(1, cam, disc, outs);
  if (st) return st;
  BH_CUDA(cudaSetDevice(ctx->device));
  std::lock_guard<std::mutex> lk(ctx->mu);
  st = serve_init(ctx);
  if (st) return st;
  Request r;
  memset(&r.job, 0, sizeof r.job);
  r.orbit = false;
  r.cam = *cam;
  return enqueue(ctx, r, t, cube, viewer, disc, sh, out, sizeof(float4) * (size_t)cam->width * cam->height,
                 ticket);
}

extern "C" bh_status bh_serve_submit_orbit(bh_ctx *ctx, const bh_tables *t, const bh_cubemap *cube,
                                           int viewer, bh_orbit *orbit_device, double dtau, int steps,
                                           int width, int height, const bh_disc *disc,
                                           const bh_shading *sh, float *out, unsigned long long *ticket) {
  if (!ctx || !t || !orbit_device || !disc || !out || !ticket) {
    set_error("bh_serve_submit_orbit: NULL argument");
    return BH_ERR_INVALID_ARG;
  }
  if (viewer < 0 || viewer > 65535) { set_error("bh_serve_submit_orbit: viewer out of 0..65535"); return BH_ERR_INVALID_ARG; }
  if (((uintptr_t)orbit_device & 7) || ((uintptr_t)out & 15)) {
    set_error("bh_serve_submit_orbit: orbit must be 8-byte and out 16-byte aligned");
    return BH_ERR_INVALID_ARG;
  }
  if (width < 1 || height < 1 || width > 16384 || height > 16384 || steps < 0 || steps > 100000 ||
      !(dtau >= 0.0) || !std::isfinite(dtau) || (steps > 0 && dtau == 0.0)) {
    set_error("bh_serve_submit_orbit: need 1..16384 pixels a side, 0 <= steps <= 100000, finite dtau >= 0");
    return BH_ERR_INVALID_ARG;
  }
  if (!validate_disc_ext(disc)) return BH_ERR_INVALID_ARG;
  BH_CUDA(cudaSetDevice(ctx->device));
  std::lock_guard<std::mutex> lk(ctx->mu);
  bh_status st = serve_init(ctx);
  if (st) return st;
  Request r;
  memset(&r.cam, 0, sizeof r.cam);
  r.orbit = true;
  r.job = OrbitJob{orbit_device, out, dtau, steps, width, height, 0};
  return enqueue(ctx, r, t, cube, viewer, disc, sh, out, sizeof(float4) * (size_t)width * height, ticket);
}

extern "C" bh_status bh_serve_poll(bh_ctx *ctx, unsigned long long ticket, int timeout_us,
                                   double *latency_ms) {
  if (!ctx) { set_error("bh_serve_poll: NULL context"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(ctx->device));
  Clock::time_point t_end = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      bh_status st = serve_init(ctx);
      if (st) return st;
      ServeState *S = ctx->serve;
      if (ticket == 0 || ticket >= S->next_ticket) { set_error("bh_serve_poll: unknown ticket"); return BH_ERR_INVALID_ARG; }
      st = progress(ctx);
      if (st) return st;
      auto it = S->finished.find(ticket);
      if (it != S->finished.end()) {
        if (latency_ms) *latency_ms = it->second;
        S->finished.erase(it);
        return BH_OK;
      }
    }
    if (Clock::now() >= t_end) return BH_ERR_NOT_READY;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

extern "C" bh_status bh_serve_flush(bh_ctx *ctx) {
  if (!ctx) { set_error("bh_serve_flush: NULL context"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(ctx->device));
  std::lock_guard<std::mutex> lk(ctx->mu);
  bh_status st = serve_init(ctx);
  if (st) return st;
  return progress(ctx);
}
