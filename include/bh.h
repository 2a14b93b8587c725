/*
 * bh.h -- C ABI of libbh, a GB300 (sm_103a) implementation of the
 * table-driven beam tracer for a non-rotating (Schwarzschild) black hole of
 * E. Bruneton, "Real-time High-Quality Rendering of Non-Rotating Black
 * Holes" (2020).
 *
 * The problem statement (Sec. 3, Sec. 4): camera position, velocity and
 * orientation, accretion-disc parameters and a star list in; a linear-RGB
 * image out.  Units: horizon radius r_s = 1 and c = 1 (Sec. 3.1).
 *
 * Conventions shared by every call:
 *  - Every call returns a bh_status; no exception or signal crosses the ABI.
 *    On failure bh_last_error() returns a message for the calling thread.
 *  - Handles (bh_ctx, bh_tables, bh_cubemap) are owned by the library and
 *    released by their _free / bh_destroy call.  Image buffers are owned by
 *    the caller.
 *  - "device" pointers are CUDA device pointers of the context's device;
 *    "host" pointers are ordinary (preferably pinned) host memory.
 *  - Streams are passed as void* holding a cudaStream_t (NULL = the legacy
 *    default stream).  Calls that take a stream only enqueue work on it
 *    unless their comment says they synchronise.
 *  - Invalid physics is rejected with BH_ERR_INVALID_ARG: camera radius
 *    r <= 1 (no static observer inside the horizon, Sec. 5), |v| >= 1, a
 *    non-orthonormal orientation, disc r_in < 3 (innermost stable circular
 *    orbit, Sec. 3.3.3) or r_out <= r_in.
 */
#ifndef BH_H
#define BH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BH_OK = 0,
  BH_ERR_INVALID_ARG = 1,   /* a pointer, size or physical parameter is out of range */
  BH_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the CUDA error) */
  BH_ERR_OOM = 3,           /* device allocation failed or the memory budget is exceeded */
  BH_ERR_BUSY = 4,          /* serving: admission refused the request */
  BH_ERR_NOT_READY = 5,     /* serving: the ticket's frame is not finished yet */
  BH_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  BH_ERR_DEVICE_STATUS = 7  /* a kernel reported an error through its status word */
} bh_status;

typedef enum { BH_F32 = 0, BH_F16 = 1, BH_BF16 = 2 } bh_dtype;

typedef struct bh_ctx bh_ctx;
typedef struct bh_tables bh_tables;
typedef struct bh_cubemap bh_cubemap;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory the serving loop may hold for frames in flight (0 = no
 * bound).  The context owns a status word, small staging buffers and, once
 * used, the serving streams. */
bh_status bh_create(int device, size_t hbm_budget_bytes, bh_ctx **out);
void bh_destroy(bh_ctx *ctx);

/* Message of the last failed call on this thread ("" if none).  Valid until
 * the next call on this thread. */
const char *bh_last_error(void);

/* Number of kernel launches the context has issued so far (all entry
 * points), for launch accounting. */
long long bh_kernel_launches(const bh_ctx *ctx);

/* Synchronise `stream` and read the context's kernel status word: BH_OK, or
 * BH_ERR_TIMEOUT if a render's bounded wait for its shared-memory tables gave
 * up (the block skipped its tiles), or BH_ERR_DEVICE_STATUS.  Clears the word. */
bh_status bh_check_status(bh_ctx *ctx, void *stream);

/* Failure detection tests: make the next render launch of this context, after
 * its tables have landed, also wait on a barrier that nothing arrives at (kind
 * BH_FAULT_TABLE_WAIT), so that its bounded wait (2 ms) runs out, the blocks
 * skip their tiles and bh_check_status reports BH_ERR_TIMEOUT; or make one
 * block of the next bloom launch never arrive at its first grid barrier (kind
 * BH_FAULT_BLOOM_BARRIER), so that every block's bounded barrier wait (2 ms)
 * runs out and the blocks stop (the output is left unfinished) and
 * bh_check_status reports BH_ERR_TIMEOUT.  The context stays usable.  No
 * fault, trap or hang is produced. */
#define BH_FAULT_TABLE_WAIT 1
#define BH_FAULT_BLOOM_BARRIER 2
bh_status bh_inject_fault(bh_ctx *ctx, int kind);

/* Issue rates of the SMs of CUDA device `device`, measured by the library's
 * own microbenchmark kernels (independent dependency chains on every SM; the
 * paper has no counterpart -- these are the denominators of the render
 * kernel's roofline).  out[0]: scalar FP32 FMA results per SM per clock;
 * out[1]: FMA results per SM per clock issued as packed f32x2 FMAs; out[2]:
 * special-function (reciprocal square root) results per SM per clock;
 * out[3]: the SM count; out[4]: the SM clock seen during the measurement, MHz.
 * out holds 5 doubles.  Synchronises the device; allocates a few bytes. */
bh_status bh_measure_issue_rates(int device, double *out);

/* Bandwidth from device memory to pinned host memory on CUDA device
 * `device`, the bound of every frame that goes to the host: `bytes` (rounded
 * down to a multiple of 16, at least 16) moved by the copy engine
 * (cudaMemcpyAsync device to pinned host, out[0]) and written into mapped
 * pinned host memory by the library's own kernel stores (whole 128-byte lines
 * per warp, out[1]), each in GB/s, the best of five timed runs after one
 * untimed.  Allocates `bytes` of device memory and of pinned host memory for
 * the call; synchronous.  BH_ERR_INVALID_ARG for a NULL out or bytes < 16. */
bh_status bh_measure_host_link(int device, size_t bytes, double *out);

/* ------------------------------------------------------------------------ */
/* Tables D(e,u), U(e,phi) (Algorithm 1 PRECOMPUTE, Sec. 3.3.2-3.3.3,        */
/* Appendix A) and the colour tables (Sec. 3.4.2)                             */
/* ------------------------------------------------------------------------ */

/* d_n x d_n deflection table D (d_n even, 4..4096; the paper uses 512) and
 * u_ne x u_nphi disc table U (the paper uses 64 x 32; u_ne * u_nphi <= 4096).
 * storage: BH_F32 or BH_F16 for the copies the renderer reads.  Texel i of n
 * holds the Appendix A coordinate i/(n-1). */
typedef struct {
  int d_n;
  int u_ne;
  int u_nphi;
  bh_dtype storage;
} bh_table_desc;

/* Compute D and U on the GPU by FP64 quadrature of the ray equation
 * (Eq. rayequation: (du/dphi)^2 = e^2 - u^2 (1-u)), one thread per texel, and
 * the colour tables: C(xy, D) (64 x 32 x 64, Sec. 3.4.2) and the black-body
 * table used for the disc.  Enqueued on `stream`; *out is usable by later
 * work on the same stream at once.  Allocates device memory (~10 MiB). */
bh_status bh_precompute_tables(bh_ctx *ctx, const bh_table_desc *desc, void *stream,
                               bh_tables **out);

/* Same handle from host FP64 values (D[j*d_n + i], U[j*u_ne + i]; i indexes
 * e, j indexes u or phi), converted to the storage type on the device; the
 * colour tables are computed on the GPU as in bh_precompute_tables.
 * Synchronises `stream`. */
bh_status bh_tables_upload(bh_ctx *ctx, const bh_table_desc *desc, const double *D_host,
                           const double *U_host, void *stream, bh_tables **out);

/* Copy the FP64 values of D and U to host buffers (d_n*d_n and
 * u_ne*u_nphi doubles; either may be NULL).  Synchronises the context's
 * device. */
bh_status bh_tables_copy_out(const bh_tables *t, double *D_host, double *U_host);

/* Retarded-time channels of D and U (Algorithm 1 stores the coordinate time
 * t beside Delta and u).  Both hold the regularised time
 *     R = t + 1/u - ln(u / (1 - u)),   dR/dphi = 1 / (e + du/dphi),
 * with t = 0 at phi = 0 (the ray's start at infinity), finite everywhere on
 * the tables (t itself diverges at u = 0 and at the horizon).  DT has D's
 * layout and texel coordinates; UT has U's, 0 where the ray was captured or
 * does not exist.  Past the apsis UT follows from t(phi) = 2 t_a -
 * t(2 phi_a - phi).  bh_precompute_tables fills them; after bh_tables_upload
 * they are NaN until bh_tables_upload_time sets them from host FP64 values
 * (same layouts; synchronises `stream`).  bh_tables_copy_time copies them
 * out (either pointer may be NULL; synchronises the device). */
bh_status bh_tables_upload_time(bh_tables *t, const double *DT_host, const double *UT_host,
                                void *stream);
bh_status bh_tables_copy_time(const bh_tables *t, double *DT_host, double *UT_host);

/* Checkpoints.  bh_tables_save writes every table of the handle (D, U and
 * their time channels in FP64, the C and black-body tables) to `path`;
 * bh_tables_load rebuilds a handle from such a file without recomputing
 * anything (synchronises `stream`).  bh_cubemap_save / bh_cubemap_load do the
 * same for a star cube map (records and occupancy mask).  Files carry a magic,
 * a format version, the sizes, the texel-coordinate convention and an FNV-1a
 * 64-bit hash of their contents; a file that is truncated, corrupt, of
 * another version or inconsistent is refused with BH_ERR_INVALID_ARG before
 * any device memory is allocated. */
bh_status bh_tables_save(const bh_tables *t, const char *path);
bh_status bh_tables_load(bh_ctx *ctx, const char *path, void *stream, bh_tables **out);
bh_status bh_cubemap_save(const bh_cubemap *c, const char *path);
bh_status bh_cubemap_load(bh_ctx *ctx, const char *path, void *stream, bh_cubemap **out);

/* Copy the colour tables: C as [log2 D][y][x] float4 (XYZ, pad), 64*32*64*4
 * floats; the disc black-body table as 1024 float4 (ln Y, X/Y, Z/Y, pad) at
 * log2 T = 8 + 12 (k + 1/2)/1024.  Either may be NULL.  Synchronises. */
bh_status bh_tables_copy_colour(const bh_tables *t, float *C_host, float *disc_host);
void bh_tables_free(bh_tables *t);

/* ------------------------------------------------------------------------ */
/* Star cube map (Sec. 3.3.2 "Emitted light", Sec. 4)                         */
/* ------------------------------------------------------------------------ */

/* A synthetic star: unit direction in the black hole's Cartesian frame,
 * luminosity (X+Y+Z of its emitted colour) and black-body temperature. */
typedef struct {
  float dir[3];
  float lum;
  float temp_K;
} bh_star;

/* Bin n stars into a 6 x face_size^2 cube map with a full mip chain: each
 * texel stores the colour sum (X, Y, Z as half or bfloat16 of the sum
 * divided by 4^level) and the luminance-weighted mean star position inside
 * the texel (two unorm8); mips sum colours and average positions weighted by
 * Y.  face_size: power of two, 1..8192.  storage: BH_F16 or BH_BF16.
 * stars: host array (stars_on_device = 0) or device array (1).  Enqueued on
 * `stream` (a host star list is staged synchronously first).  Uses
 * 40 * 6 * face_size^2 bytes of scratch, freed before return. */
bh_status bh_build_star_cubemap(bh_ctx *ctx, const bh_star *stars, long long n, int face_size,
                                bh_dtype storage, int stars_on_device, void *stream,
                                bh_cubemap **out);

/* Allocation-free form of bh_build_star_cubemap, for callers that may not
 * allocate device memory themselves (applications that give all device
 * memory to their own pool or arena, real-time threads that must not call
 * cudaMalloc/cudaFree because those can synchronise the device).  The paper
 * has no counterpart; the records are the same as bh_build_star_cubemap's.
 *  - stars_device: n stars in device memory; records_device: caller-owned
 *    device buffer of bh_cubemap_records(face_size) x 4 uint16, 8-byte aligned.
 *  - face_size: power of two, at most 128 (the size of the library's static
 *    scratch array, about 6.9 MB, held on every GPU that loads the library
 *    until the process exits); larger sizes return BH_ERR_INVALID_ARG.
 *  - Works on the current CUDA device and needs no bh_ctx; `stream`, the
 *    stars and the records must all belong to that device.  Each call that is
 *    not under stream capture looks up the scratch array's device address on
 *    that device; a call under capture reuses the address the device's last
 *    uncaptured call found, so make one call before capturing (a first call
 *    under capture returns BH_ERR_INVALID_ARG).
 *  - Allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 *    Every call shares the one scratch array, so calls whose work overlaps
 *    on the GPU (other streams, other threads) race: serialise them.
 *  - Enqueued on `stream`. */
bh_status bh_build_star_cubemap_noalloc(const bh_star *stars_device, long long n, int face_size,
                                        bh_dtype storage, uint16_t *records_device, void *stream);

/* Number of texel records (all faces, all levels) of a cube map. */
long long bh_cubemap_records(int face_size);

/* Copy all records (4 uint16 per texel, level-major, face, row, column) to
 * the host; n_records must equal bh_cubemap_records(face_size).  Synchronises. */
bh_status bh_cubemap_copy_out(const bh_cubemap *c, uint16_t *records_host, long long n_records);
void bh_cubemap_free(bh_cubemap *c);

/* ------------------------------------------------------------------------ */
/* Rendering (Sec. 3.2-3.4, Algorithm 1 TRACERAY)                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  double r, theta, phi; /* Schwarzschild position, r > 1 */
  double v[3];          /* velocity wrt the static observer, components on (e_r, e_theta, e_phi), |v| < 1 */
  double orient[9];     /* O, row-major: rows e_w, e_h, e_d on the boosted (r', theta', phi') axes */
  double fov_y;         /* vertical field of view, radians, in (0, pi) */
  int width, height;    /* pixels, 1..16384 each */
} bh_camera;

typedef struct bh_particles bh_particles;

typedef struct {
  double r_in, r_out; /* 3 <= r_in < r_out; disc in the z = 0 plane, prograde about +z */
  double t_peak_K;    /* temperature at r = 49/12, where T^4 ~ u^3 (1 - sqrt(3u)) peaks */
  double density;     /* in [0,1]: emission weight and opacity of each disc crossing */
  int enabled;
  /* Animated disc (Appendix B), or NULL for the constant density above.  With
   * particles, the density of a crossing is min(1, density * sum_p f_p), f_p
   * the contribution of linear particle p at the crossing's retarded time
   * time - delay (delay from the tables' time channels, which must be set),
   * radius and azimuth. */
  const bh_particles *particles;
  double time;        /* coordinate time of the frame at the camera */
} bh_disc;

/* Linear particles of the animated disc (Appendix B): n rows of 3 doubles
 * (u1, u2, phi0), 0 < u1 <= u2 <= 1/3, 1 <= n <= 256.  Each row is a
 * quasi-circular precessing orbit, phi(t) = sqrt(ubar^3/2) t + phi0 with
 * ubar = (u1 + u2)/2, u(phi) = u1 + (u2 - u1) sin^2(pi/(4K) phi sqrt(u3 - u1)),
 * u3 = 1 - u1 - u2, K the complete elliptic integral of the first kind of
 * modulus sqrt((u2 - u1)/(u3 - u1)).  A crossing at time t, radius r and
 * azimuth phi takes a = (phi - phi(t)) mod 2 pi, d^2 = (a/pi - 1)^2 +
 * (r - 1/u(a + phi(t)))^2 and f = (1 - d^2)^2 for d < 1, else 0.  The rows
 * are copied to device memory (sorted by radius); invalid rows give
 * BH_ERR_INVALID_ARG. */
bh_status bh_disc_particles_create(bh_ctx *ctx, const double *particles_host, int n,
                                   bh_particles **out);
void bh_disc_particles_free(bh_particles *p);

typedef struct {
  float exposure_disc;  /* disc radiance scale: 1 = peak black body of Y = 1 */
  float exposure_stars; /* star radiance scale */
} bh_shading;

/* Render one frame: out_rgba_device holds width*height float4 (linear sRGB,
 * A = 1), row-major, top row first; caller-owned device memory, 16-byte
 * aligned.  cubemap may be NULL (no stars).  Enqueued on `stream`. */
bh_status bh_render(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                    const bh_camera *camera, const bh_disc *disc, const bh_shading *shading,
                    float *out_rgba_device, void *stream);

/* As bh_render, plus 20 floats per pixel of intermediate values in
 * dbg_device (16-byte aligned): e^2, delta, delta' (+inf if captured),
 * number of disc hits, u0, u1, mip level (-1: no star term), cube face,
 * Omega/Omega', star Doppler factor, gathered star X, Y, Z, hit-0 Doppler,
 * hit-1 Doppler, texels visited, then the retarded-time delays of hits 0
 * and 1 (coordinate time from the disc point to the camera along the beam,
 * from the tables' time channels; 0 without a hit) and the disc densities
 * of hits 0 and 1 (0 without a hit).  The debug render is also a checked
 * build: every table, cube-map and occupancy index is tested before its
 * access; an index out of range skips the access and makes bh_check_status
 * return BH_ERR_DEVICE_STATUS. */
bh_status bh_render_debug(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                          const bh_camera *camera, const bh_disc *disc,
                          const bh_shading *shading, float *out_rgba_device, float *dbg_device,
                          void *stream);

/* End-to-end form: the image lands in out_rgba_host (width*height*4 floats).
 * Pinned memory the device can address is written by the kernel directly
 * (the transfer overlaps the rendering); other memory receives a copy of a
 * context-owned device frame.  Synchronises `stream` before returning. */
bh_status bh_render_to_host(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                            const bh_camera *camera, const bh_disc *disc,
                            const bh_shading *shading, float *out_rgba_host, void *stream);

/* As bh_render_to_host, with the image as packed linear RGB: width*height*3
 * floats, row-major, top row first (the alpha channel, always 1, is not
 * sent: a quarter less over the host link).  Pinned memory the device can
 * address is written by the kernel directly; when it is 16-byte aligned and
 * width % 4 == 0, every warp stores its four 96-byte pixel-row runs as
 * 16-byte chunks.  Synchronises `stream` before returning. */
bh_status bh_render_to_host_rgb(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                                const bh_camera *camera, const bh_disc *disc,
                                const bh_shading *shading, float *out_rgb_host, void *stream);

/* Frames to the host with two in flight: renders the frame into one of two
 * context-owned device frames on `stream` and returns at once; the copy
 * engine then moves it into out_host on a context-owned copy stream while
 * the next call's frame renders into the other device frame (a device frame
 * is rendered into again only after its previous copy has finished).
 *  - out_host: pinned host memory (cudaHostAlloc, cudaHostRegister) of
 *    width*height*4 floats (rgb = 0: RGBA as bh_render) or width*height*3
 *    (rgb = 1: packed linear RGB as bh_render_to_host_rgb); it must stay
 *    allocated and unread until bh_host_wait(ticket) returns.
 *  - *ticket receives the frame's number (0, 1, 2, ... per context).
 * Errors: BH_ERR_INVALID_ARG for NULL arguments, an invalid camera, rgb not
 * 0 or 1, or pageable out_host (nothing is enqueued then).  The image is the
 * one bh_render / bh_render_to_host_rgb produce for the same arguments. */
bh_status bh_render_to_host_async(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                                  const bh_camera *camera, const bh_disc *disc,
                                  const bh_shading *shading, float *out_host, int rgb, void *stream,
                                  unsigned long long *ticket);

/* Block until frame `ticket` of bh_render_to_host_async is in host memory
 * (it may return after a later frame's copy, which implies this one's).
 * BH_ERR_INVALID_ARG for a ticket that was never issued. */
bh_status bh_host_wait(bh_ctx *ctx, unsigned long long ticket);

/* Render n cameras of any sizes in one persistent launch driven by a tile
 * queue: outs[k] is camera k's device image (as bh_render).  The per-camera
 * constants are staged through the context.  Enqueued on `stream`. */
bh_status bh_render_batch(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap, int n,
                          const bh_camera *cameras, const bh_disc *disc,
                          const bh_shading *shading, float *const *outs, void *stream);

/* Autotuning of the batched launch: time the candidate launch shapes on the
 * given cameras (renders them several times, synchronously, each timed run
 * from a cold L2: a temporary scratch buffer of twice the L2 size is cleared
 * before it; timed warm if that buffer cannot be allocated) and keep the
 * shape with the smallest median time for later bh_render_batch calls of this
 * context.  *chosen receives the chosen candidate index (may be NULL). */
bh_status bh_autotune_batch(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                            int n, const bh_camera *cameras, const bh_disc *disc,
                            const bh_shading *shading, float *const *outs, int *chosen);

/* ------------------------------------------------------------------------ */
/* Lens glare (Sec. 3.4.3)                                                    */
/* ------------------------------------------------------------------------ */

/* Weights of the bloom's levels for a camera of vertical field of view fov_y
 * (radians) and `height` pixels: weights[k] (k = 0..levels, levels <= 10) is
 * the share of the photopic point spread function of Spencer et al. (1995),
 *   P(theta) = 0.384 f0 + 0.478 f1 + 0.138 f2 (theta in degrees),
 *   f0 = 2.61e6 exp(-(theta/0.02)^2), f1 = 20.91/(theta+0.02)^3,
 *   f2 = 72.37/(theta+0.02)^2,
 * falling between radii 2^(k-1/2) and 2^(k+1/2) pixels (k = 0: below
 * 2^(1/2)), out of its energy below 2^(levels+1/2) pixels (pixel angle =
 * fov_y / height).  The weights sum to 1.  Host only. */
bh_status bh_bloom_weights(double fov_y, int height, int levels, double *weights);

/* Bloom of a linear-RGB frame before tone mapping (Sec. 3.4.3: small filter
 * kernels on mipmaps of the image approximating the PSF above).  in_device,
 * out_device: width*height float4 (RGB, A = 1), 16-byte aligned; they may be
 * the same buffer.  D_0 = in; D_k = 2x2 box average of D_{k-1} (sizes rounded
 * up, indices clamped); B_k = D_k blurred by a separable 7-tap Gaussian of unit
 * standard deviation (clamped); out = weights[0] in + sum_k weights[k]
 * bilinear(B_k) at the pixel centre (clamped), k = 1..levels (<= 10).  The
 * pyramid lives in context-owned scratch (allocated on first use, grown as
 * needed), so bloom calls of one context must not overlap on the GPU
 * (enqueue them on one stream).  Enqueued on `stream`. */
bh_status bh_bloom(bh_ctx *ctx, const float *in_device, float *out_device, int width, int height,
                   int levels, const double *weights, void *stream);

/* ------------------------------------------------------------------------ */
/* Free-fall camera orbits (Appendix C), resident on the device               */
/* ------------------------------------------------------------------------ */

/* A camera on a geodesic: coordinate time t, radius r and angle psi in an
 * orbital plane of inclination chi (position r (cos chi cos psi, sin psi,
 * sin chi cos psi)), dr/dtau, and the constants of motion e, l.  orient: the
 * user rotation O, rows e_w, e_h, e_d on the boosted (r', chi', psi') axes. */
typedef struct {
  double t, r, psi, rdot;
  double e, l;
  double chi;
  double orient[9];
  double fov_y;
  int width, height;
} bh_orbit;

/* Initial state from the radius r0 > 1.05, the angle delta0 in (0, pi) of the
 * velocity from the radius (tan delta = r dpsi/dr) and the speed v0 in [0,1)
 * wrt the static observer: e^2 = (1-u0)/(1-v0^2), l^2 = (e^2+u0-1) /
 * (u0^2 (1-u0+cot^2 delta0)) (Appendix C).  orient may be NULL (identity). */
bh_status bh_orbit_init(double r0, double delta0, double v0, double chi, const double *orient,
                        double fov_y, int width, int height, bh_orbit *out);

/* The camera (position, velocity wrt the static observer, orientation on the
 * boosted (r', theta', phi') axes) of an orbit state; host only. */
bh_status bh_orbit_camera(const bh_orbit *orbit, bh_camera *out);

/* Advance n device-resident orbits by dtau of proper time in `steps` FP64
 * Runge-Kutta steps of d^2r/dtau^2 = (2 l^2 u^3 - 3 l^2 u^4 - u^2)/2,
 * dpsi/dtau = l u^2, dt/dtau = e/(1-u).  An orbit that would reach r <= 1.05
 * stops there.  Enqueued on `stream`. */
bh_status bh_orbits_advance(bh_ctx *ctx, bh_orbit *orbits_device, int n, double dtau, int steps,
                            void *stream);

/* Render n <= 1024 device-resident orbits in one persistent launch: their
 * camera constants are computed on the device (no host round trip); outs[k]
 * as in bh_render_batch.  Enqueued on `stream`. */
bh_status bh_render_orbits(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap, int n,
                           const bh_orbit *orbits_device, const bh_disc *disc,
                           const bh_shading *shading, float *const *outs, void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of frame requests from many viewers          */
/* ------------------------------------------------------------------------ */

/* Submit a frame request of viewer `viewer` (0..65535) into a caller-owned
 * device buffer.  Requests are batched with those already queued and start
 * as soon as a launch slot frees; admission is refused with BH_ERR_BUSY if
 * the frame does not fit the context's memory budget or the viewer already
 * has a frame queued (reading: at most one queued and one in flight per
 * viewer).  *ticket identifies the request for bh_serve_poll. */
bh_status bh_serve_submit(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                          int viewer, const bh_camera *camera, const bh_disc *disc,
                          const bh_shading *shading, float *out_rgba_device,
                          unsigned long long *ticket);

/* Serving viewers on device-resident orbits (Appendix C): the request of
 * `viewer` advances its orbit (*orbit_device: caller-owned device memory, one
 * bh_orbit per viewer, 8-byte aligned) by dtau of proper time in `steps`
 * Runge-Kutta steps on the device (steps = 0: no advance), as
 * bh_orbits_advance does, then renders it at width x height into out_device
 * (16-byte aligned, width*height*4 floats; the orbit's own size fields are
 * ignored).  Batching, admission and polling as bh_serve_submit; requests of
 * one viewer advance its orbit in submission order even when consecutive
 * batches run on different streams. */
bh_status bh_serve_submit_orbit(bh_ctx *ctx, const bh_tables *tables, const bh_cubemap *cubemap,
                                int viewer, bh_orbit *orbit_device, double dtau, int steps, int width,
                                int height, const bh_disc *disc, const bh_shading *shading,
                                float *out_device, unsigned long long *ticket);

/* Progress the serving loop and report on a ticket: BH_OK when its frame is
 * finished (latency_ms = submit to completion), BH_ERR_NOT_READY while
 * pending (waits up to timeout_us microseconds first; 0 = do not wait).
 * The serving loop has no thread of its own: queued requests are launched
 * only inside bh_serve_submit, bh_serve_submit_orbit, bh_serve_poll and
 * bh_serve_flush.  A client that submits and then stops calling leaves its
 * queued (not yet launched) frames waiting; poll or flush to keep work
 * moving. */
bh_status bh_serve_poll(bh_ctx *ctx, unsigned long long ticket, int timeout_us,
                        double *latency_ms);

/* Launch whatever is queued without waiting for more requests. */
bh_status bh_serve_flush(bh_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BH_H */
