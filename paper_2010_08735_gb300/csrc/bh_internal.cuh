// Internal declarations shared by the libbh translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bh.h"

namespace bh {

// NVTX range over a C-ABI call (precompute, cube map, render, batch, serve):
// visible in a profiler's timeline, free when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

constexpr double kMu = 4.0 / 27.0;  // max of u^2 (1-u), photon sphere u = 2/3 (Sec. 3.3.1)
constexpr double kPi = 3.14159265358979323846;

// Sizes of the colour tables (Sec. 3.4.2 and the disc black-body table).
constexpr int kCnx = 64, kCny = 32, kCnd = 64;
constexpr int kDiscN = 1024;
constexpr int kNLambda = 95;  // 360..830 nm, 5 nm trapezoid
constexpr int kNLocus = 4096;
constexpr int kMaxUTexels = 4096;
constexpr int kMaxParticles = 256;  // animated disc: shared memory holds 32 bytes per particle

// Status word bits written by kernels (never a trap or an assert).
constexpr unsigned kStatusMbarTimeout = 1u;
constexpr unsigned kStatusBadIndex = 2u;
constexpr unsigned kStatusBarrierTimeout = 4u;  // a bounded grid-barrier wait gave up

void set_error(const char *fmt, ...);
bh_status cuda_fail(cudaError_t e, const char *what);
#define BH_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

struct ServeState;

// A batched launch as a CUDA graph: the copy of the per-camera constants
// from pinned staging memory and the persistent render kernel.  Rebuilt when
// the number of cameras or the kernel changes; otherwise only the kernel's
// parameters are updated before each replay.
struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t copy = nullptr, kern = nullptr;
  int n = 0, block = 0;
  const void *func = nullptr;
  void *cam_dev = nullptr;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    copy = kern = nullptr;
    n = block = 0;
    func = nullptr;
    cam_dev = nullptr;
  }
};

struct RenderTuning {
  int warps_per_block = 8;   // block = warps * 32 threads
  int fetch = 2;             // 8 x 4 pixel warp tiles a warp takes per fetch
  int blocks_per_sm = 4;     // persistent grid = SMs * blocks_per_sm
};

// A served frame request on a device-resident orbit (Appendix C): advance
// *orbit by dtau of proper time in `steps` steps, then render it at
// width x height into out.
struct OrbitJob {
  bh_orbit *orbit;
  float *out;
  double dtau;
  int steps, width, height, pad;
};

// Tile-scheduler counters: every render launch takes the next pair of a ring
// (re-armed to zero by the launch's last warp), so launches in flight at once
// on different streams need distinct pairs: at most kSchedRing of them.
constexpr int kSchedRing = 1024;

}  // namespace bh

struct bh_ctx {
  int device = 0;
  int sm_count = 0;
  size_t budget = 0;
  cudaStream_t aux = nullptr;
  unsigned *status_dev = nullptr;     // kernel status word
  unsigned *sched_dev = nullptr;      // kSchedRing pairs of tile-scheduler counters
  std::atomic<unsigned> sched_next{0};
  std::atomic<long long> launches{0};
  // render staging: per-camera constants for batched launches
  void *cam_host = nullptr;           // pinned
  void *cam_dev = nullptr;
  int cam_cap = 0;
  bh::BatchGraph graph;               // bh_render_batch launches
  void *orb_outs_host = nullptr;      // bh_render_orbits: pinned output pointers
  void *orb_outs_dev = nullptr;       // device copy of them, then the tile count
  void *orb_cams_dev = nullptr;       // per-orbit camera constants
  int orb_cap = 0;
  float *frame_dev = nullptr;         // bh_render_to_host frame buffer
  size_t frame_cap = 0;
  // bh_render_to_host_async: two device frames; each is copied to the host
  // on ring_copy while the next one renders
  float *ring_dev[2] = {nullptr, nullptr};
  size_t ring_cap = 0;
  cudaStream_t ring_copy = nullptr;
  cudaEvent_t ring_ready[2] = {nullptr, nullptr};  // the slot's last frame is rendered
  cudaEvent_t ring_done[2] = {nullptr, nullptr};   // ... and its copy to the host has finished
  unsigned long long ring_seq = 0;                 // frames issued (the next ticket)
  void *bloom_dev = nullptr;          // bh_bloom: mip pyramid scratch
  size_t bloom_cap = 0;
  unsigned *bloom_bar = nullptr;      // bh_bloom: grid-barrier counter
  bh::RenderTuning tuning;
  bh::ServeState *serve = nullptr;
  int inject_table_wait = 0;          // bh_inject_fault: next render's table wait never completes
  int inject_bloom_barrier = 0;       // bh_inject_fault: next bloom's first grid barrier is never complete
  std::mutex mu;
};

struct bh_tables {
  bh_ctx *ctx = nullptr;
  bh_table_desc desc{};
  double *D64 = nullptr, *U64 = nullptr;  // FP64 values
  void *D = nullptr, *U = nullptr;        // storage copies read by the renderer
  double *DT64 = nullptr, *UT64 = nullptr;  // regularised-time channels of D and U (FP64)
  float *DT = nullptr, *UT = nullptr;       // their FP32 copies (read by the debug render)
  float4 *C = nullptr;                    // colour shift table [k][j][i] (XYZ, pad)
  float4 *disc = nullptr;                 // ln Y, X/Y, Z/Y of black bodies, log2 T in [8, 20]
};

struct bh_particles {
  bh_ctx *ctx = nullptr;
  int n = 0;
  double *dev = nullptr;  // 8 doubles per particle, sorted by rmin: u1, u2, phi0, omega, c, rmin, rmax, 0
};

struct bh_cubemap {
  bh_ctx *ctx = nullptr;
  int n = 0;        // face size
  int levels = 0;
  bh_dtype storage = BH_F16;
  uint2 *rec = nullptr;  // all levels
  long long records = 0;
  unsigned *mask = nullptr;  // occupancy bits: one per texel, rows padded to 32-bit words
  long long mask_words = 0;
};

namespace bh {
inline long long cube_level_offset(int N, int L) {
  long long off = 0;
  for (int l = 0; l < L; ++l) off += 6LL * (N >> l) * (N >> l);
  return off;
}
// Occupancy mask layout: level-major, face, row; a row of n texels takes
// (n + 31) / 32 words, bit (i & 31) of word i / 32 is texel i.
inline long long mask_level_offset(int N, int L) {
  long long off = 0;
  for (int l = 0; l < L; ++l) {
    long long n = N >> l;
    off += 6LL * n * ((n + 31) / 32);
  }
  return off;
}
inline int cube_levels(int N) {
  int L = 0;
  while ((1 << L) < N) ++L;
  return L + 1;
}
void count_launch(bh_ctx *ctx, int n = 1);
bh_status check_status(bh_ctx *ctx, cudaStream_t s);
bh_status colour_tables_launch(bh_ctx *ctx, bh_tables *t, cudaStream_t s);
}  // namespace bh
