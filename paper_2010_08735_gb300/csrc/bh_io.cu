// Checkpoints of the precomputed state: tables and star cube maps saved to
// disk and loaded back without recomputation.
//
// File layout (little-endian): an 8-byte magic, a fixed header of 32-bit
// fields (format version, sizes, storage type, the texel-coordinate
// convention of the tables), the payload arrays in a fixed order, and an
// FNV-1a 64-bit hash of every preceding byte.  A load checks the magic, the
// version, the sizes against the file length and the hash before it
// allocates anything on the device.
#include <cstdio>
#include <cstring>
#include <vector>

#include "bh_internal.cuh"

namespace bh {

bh_status tables_alloc_public(bh_ctx *ctx, const bh_table_desc *desc, bh_tables **out);
bh_status tables_convert_storage(bh_ctx *ctx, bh_tables *t, cudaStream_t s);
bh_status cubemap_alloc_public(bh_ctx *ctx, int N, bh_dtype storage, bh_cubemap **out);

namespace {

constexpr char kTablesMagic[8] = {'B', 'H', 'T', 'A', 'B', 'L', 'E', 'S'};
constexpr char kCubeMagic[8] = {'B', 'H', 'C', 'U', 'B', 'E', 'M', 'P'};
constexpr uint32_t kFormatVersion = 1;
constexpr uint32_t kTexelEndpoints = 1;  // texel i of n holds the coordinate i/(n-1)

// FNV-1a, 64-bit (offset basis 14695981039346656037, prime 1099511628211).
struct Fnv1a {
  uint64_t h = 14695981039346656037ull;
  void add(const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

struct Writer {
  FILE *f = nullptr;
  Fnv1a hash;
  bool ok = true;
  explicit Writer(const char *path) : f(fopen(path, "wb")) { ok = f != nullptr; }
  ~Writer() {
    if (f) fclose(f);
  }
  void put(const void *p, size_t n) {
    if (!ok) return;
    hash.add(p, n);
    ok = fwrite(p, 1, n, f) == n;
  }
  bool finish() {
    if (!ok) return false;
    uint64_t h = hash.h;
    ok = fwrite(&h, 1, sizeof h, f) == sizeof h;
    ok = fclose(f) == 0 && ok;
    f = nullptr;
    return ok;
  }
};

// Whole file in memory, hash verified; get() walks the payload.
struct Reader {
  std::vector<unsigned char> buf;
  size_t pos = 0;
  bool load(const char *path) {
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    fseek(f, 0, SEEK_END);
    long n = ftell(f);
    fseek(f, 0, SEEK_SET);
    if (n < 16) {
      fclose(f);
      return false;
    }
    buf.resize((size_t)n);
    bool ok = fread(buf.data(), 1, buf.size(), f) == buf.size();
    fclose(f);
    return ok;
  }
  bool hash_ok() const {
    Fnv1a h;
    h.add(buf.data(), buf.size() - 8);
    uint64_t stored;
    memcpy(&stored, buf.data() + buf.size() - 8, 8);
    return stored == h.h;
  }
  size_t payload() const { return buf.size() - 8; }
  bool get(void *p, size_t n) {
    if (pos + n > payload()) return false;
    memcpy(p, buf.data() + pos, n);
    pos += n;
    return true;
  }
  const unsigned char *take(size_t n) {
    if (pos + n > payload()) return nullptr;
    const unsigned char *p = buf.data() + pos;
    pos += n;
    return p;
  }
};

template <typename T>
bh_status copy_out(std::vector<T> &v, const void *dev, size_t n) {
  v.resize(n);
  BH_CUDA(cudaMemcpy(v.data(), dev, sizeof(T) * n, cudaMemcpyDeviceToHost));
  return BH_OK;
}

}  // namespace
}  // namespace bh

using namespace bh;

extern "C" bh_status bh_tables_save(const bh_tables *t, const char *path) {
  TraceRange trace_("bh_tables_save");
  if (!t || !path) { set_error("bh_tables_save: NULL argument"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(t->ctx->device));
  BH_CUDA(cudaDeviceSynchronize());
  const size_t nd = (size_t)t->desc.d_n * t->desc.d_n, nu = (size_t)t->desc.u_ne * t->desc.u_nphi;
  std::vector<double> D, U, DT, UT;
  std::vector<float4> Cc, disc;
  bh_status st;
  if ((st = copy_out(D, t->D64, nd)) || (st = copy_out(U, t->U64, nu)) || (st = copy_out(DT, t->DT64, nd)) ||
      (st = copy_out(UT, t->UT64, nu)) || (st = copy_out(Cc, t->C, (size_t)kCnx * kCny * kCnd)) ||
      (st = copy_out(disc, t->disc, (size_t)kDiscN)))
    return st;
  Writer w(path);
  const uint32_t hdr[8] = {kFormatVersion, (uint32_t)t->desc.d_n, (uint32_t)t->desc.u_ne, (uint32_t)t->desc.u_nphi,
                           (uint32_t)t->desc.storage, kTexelEndpoints, (uint32_t)(kCnx * kCny * kCnd),
                           (uint32_t)kDiscN};
  w.put(kTablesMagic, 8);
  w.put(hdr, sizeof hdr);
  w.put(D.data(), nd * 8);
  w.put(U.data(), nu * 8);
  w.put(DT.data(), nd * 8);
  w.put(UT.data(), nu * 8);
  w.put(Cc.data(), Cc.size() * sizeof(float4));
  w.put(disc.data(), disc.size() * sizeof(float4));
  if (!w.finish()) { set_error("bh_tables_save: cannot write %s", path); return BH_ERR_INVALID_ARG; }
  return BH_OK;
}

extern "C" bh_status bh_tables_load(bh_ctx *ctx, const char *path, void *stream, bh_tables **out) {
  TraceRange trace_("bh_tables_load");
  if (!ctx || !path || !out) { set_error("bh_tables_load: NULL argument"); return BH_ERR_INVALID_ARG; }
  *out = nullptr;
  Reader r;
  if (!r.load(path)) { set_error("bh_tables_load: cannot read %s", path); return BH_ERR_INVALID_ARG; }
  char magic[8];
  uint32_t hdr[8];
  if (!r.get(magic, 8) || memcmp(magic, kTablesMagic, 8) != 0 || !r.get(hdr, sizeof hdr)) {
    set_error("bh_tables_load: %s is not a tables file", path);
    return BH_ERR_INVALID_ARG;
  }
  if (!r.hash_ok()) { set_error("bh_tables_load: %s fails its hash (corrupt or truncated)", path); return BH_ERR_INVALID_ARG; }
  if (hdr[0] != kFormatVersion || hdr[5] != kTexelEndpoints || hdr[6] != (uint32_t)(kCnx * kCny * kCnd) ||
      hdr[7] != (uint32_t)kDiscN) {
    set_error("bh_tables_load: %s has format %u / convention %u, not %u / %u", path, hdr[0], hdr[5],
              kFormatVersion, kTexelEndpoints);
    return BH_ERR_INVALID_ARG;
  }
  bh_table_desc desc{(int)hdr[1], (int)hdr[2], (int)hdr[3], (bh_dtype)hdr[4]};
  if (desc.d_n < 4 || desc.d_n > 4096 || desc.u_ne < 2 || desc.u_nphi < 2 ||
      (size_t)desc.u_ne * desc.u_nphi > (size_t)kMaxUTexels || (desc.storage != BH_F32 && desc.storage != BH_F16)) {
    set_error("bh_tables_load: %s has invalid sizes", path);
    return BH_ERR_INVALID_ARG;
  }
  const size_t nd = (size_t)desc.d_n * desc.d_n, nu = (size_t)desc.u_ne * desc.u_nphi;
  const size_t nc = (size_t)kCnx * kCny * kCnd;
  const unsigned char *D = r.take(nd * 8), *U = r.take(nu * 8), *DT = r.take(nd * 8), *UT = r.take(nu * 8);
  const unsigned char *Cc = r.take(nc * sizeof(float4)), *disc = r.take((size_t)kDiscN * sizeof(float4));
  if (!D || !U || !DT || !UT || !Cc || !disc || r.pos != r.payload()) {
    set_error("bh_tables_load: %s has the wrong length for its sizes", path);
    return BH_ERR_INVALID_ARG;
  }
  BH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  bh_tables *t = nullptr;
  bh_status st = tables_alloc_public(ctx, &desc, &t);
  if (st) return st;
  cudaError_t e = cudaMemcpyAsync(t->D64, D, nd * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->U64, U, nu * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->DT64, DT, nd * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->UT64, UT, nu * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->C, Cc, nc * sizeof(float4), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->disc, disc, (size_t)kDiscN * sizeof(float4), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    bh_tables_free(t);
    return cuda_fail(e, "bh_tables_load");
  }
  st = tables_convert_storage(ctx, t, s);
  if (st == BH_OK) {
    e = cudaStreamSynchronize(s);  // the host buffer goes away on return
    if (e != cudaSuccess) st = cuda_fail(e, "bh_tables_load");
  }
  if (st) {
    bh_tables_free(t);
    return st;
  }
  *out = t;
  return BH_OK;
}

extern "C" bh_status bh_cubemap_save(const bh_cubemap *c, const char *path) {
  TraceRange trace_("bh_cubemap_save");
  if (!c || !path) { set_error("bh_cubemap_save: NULL argument"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(c->ctx->device));
  BH_CUDA(cudaDeviceSynchronize());
  std::vector<uint2> rec;
  std::vector<unsigned> mask;
  bh_status st;
  if ((st = copy_out(rec, c->rec, (size_t)c->records)) || (st = copy_out(mask, c->mask, (size_t)c->mask_words)))
    return st;
  Writer w(path);
  const uint32_t hdr[8] = {kFormatVersion, (uint32_t)c->n, (uint32_t)c->levels, (uint32_t)c->storage,
                           (uint32_t)(c->records & 0xffffffffu), (uint32_t)(c->records >> 32),
                           (uint32_t)(c->mask_words & 0xffffffffu), (uint32_t)(c->mask_words >> 32)};
  w.put(kCubeMagic, 8);
  w.put(hdr, sizeof hdr);
  w.put(rec.data(), rec.size() * sizeof(uint2));
  w.put(mask.data(), mask.size() * sizeof(unsigned));
  if (!w.finish()) { set_error("bh_cubemap_save: cannot write %s", path); return BH_ERR_INVALID_ARG; }
  return BH_OK;
}

extern "C" bh_status bh_cubemap_load(bh_ctx *ctx, const char *path, void *stream, bh_cubemap **out) {
  TraceRange trace_("bh_cubemap_load");
  if (!ctx || !path || !out) { set_error("bh_cubemap_load: NULL argument"); return BH_ERR_INVALID_ARG; }
  *out = nullptr;
  Reader r;
  if (!r.load(path)) { set_error("bh_cubemap_load: cannot read %s", path); return BH_ERR_INVALID_ARG; }
  char magic[8];
  uint32_t hdr[8];
  if (!r.get(magic, 8) || memcmp(magic, kCubeMagic, 8) != 0 || !r.get(hdr, sizeof hdr)) {
    set_error("bh_cubemap_load: %s is not a cube-map file", path);
    return BH_ERR_INVALID_ARG;
  }
  if (!r.hash_ok()) { set_error("bh_cubemap_load: %s fails its hash (corrupt or truncated)", path); return BH_ERR_INVALID_ARG; }
  const int N = (int)hdr[1];
  const bh_dtype storage = (bh_dtype)hdr[3];
  const long long records = (long long)hdr[4] | ((long long)hdr[5] << 32);
  const long long words = (long long)hdr[6] | ((long long)hdr[7] << 32);
  if (hdr[0] != kFormatVersion || N < 1 || N > 8192 || (N & (N - 1)) || (int)hdr[2] != cube_levels(N) ||
      (storage != BH_F16 && storage != BH_BF16) || records != cube_level_offset(N, cube_levels(N)) ||
      words != mask_level_offset(N, cube_levels(N))) {
    set_error("bh_cubemap_load: %s has an unknown format or inconsistent sizes", path);
    return BH_ERR_INVALID_ARG;
  }
  const unsigned char *rec = r.take((size_t)records * sizeof(uint2));
  const unsigned char *mask = r.take((size_t)words * sizeof(unsigned));
  if (!rec || !mask || r.pos != r.payload()) {
    set_error("bh_cubemap_load: %s has the wrong length for its sizes", path);
    return BH_ERR_INVALID_ARG;
  }
  BH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  bh_cubemap *c = nullptr;
  bh_status st = cubemap_alloc_public(ctx, N, storage, &c);
  if (st) return st;
  cudaError_t e = cudaMemcpyAsync(c->rec, rec, (size_t)records * sizeof(uint2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->mask, mask, (size_t)words * sizeof(unsigned), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    bh_cubemap_free(c);
    return cuda_fail(e, "bh_cubemap_load");
  }
  *out = c;
  return BH_OK;
}
