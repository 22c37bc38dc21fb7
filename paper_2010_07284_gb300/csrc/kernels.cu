// Plain per-operator kernels: one launch per primitive over a whole image.
// They are the baseline execution form and the building blocks of vl_ccl.
#include <algorithm>
#include <mutex>

#include "dev_ccl.cuh"
#include "dev_common.cuh"
#include "dev_select.cuh"
#include "kernels.h"

namespace vl {

namespace {

constexpr int kThreads = 256;

int grid_for(long long items, int per_block, int cap = 152 * 32) {
  long long b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// ------------------------------------------------------------ pointwise --

// A lane loads 4 pixels (16 bytes); the 8 lanes of a 32-pixel word merge
// their 4-bit pieces with three shuffles; each warp keeps two loads in flight.
__global__ void k_threshold(const void* __restrict__ plane, int format, int pitch, MaskGeom g,
                            float t, const float* t_dev, int lt, uint32_t* __restrict__ out) {
  if (t_dev) t = *t_dev;
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const long long nwords = (long long)g.H * g.Wp;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (long long base = wid * 8; base < nwords; base += nwarps * 8) {
    float4 v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long long i = base + 4 * u + (lane >> 3);
      if (i < nwords) {
        int y, w;
        split_index(i, g.Wp, y, w);
        v[u] = ld_px4(plane, format, true, (size_t)y * pitch + 32 * w + 4 * sub);
      } else {
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      uint32_t nib;
      if (lt) nib = (v[u].x < t) | ((v[u].y < t) << 1) | ((v[u].z < t) << 2) | ((v[u].w < t) << 3);
      else nib = (v[u].x > t) | ((v[u].y > t) << 1) | ((v[u].z > t) << 2) | ((v[u].w > t) << 3);
      uint32_t word = nib << (4 * sub);
      word |= __shfl_xor_sync(FULL, word, 1);
      word |= __shfl_xor_sync(FULL, word, 2);
      word |= __shfl_xor_sync(FULL, word, 4);
      const long long i = base + 4 * u + (lane >> 3);
      if (sub == 0 && i < nwords) {
        int y, w;
        split_index(i, g.Wp, y, w);
        out[i] = word & vmask(w, g.W);
      }
    }
  }
}

template <int OP>  // 0 not, 1 and, 2 or, 3 const false, 4 const true, 5 and-not
__global__ void k_pointwise(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                            MaskGeom g, uint32_t* __restrict__ out) {
  const long long nwords = (long long)g.H * g.Wp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (long long)gridDim.x * blockDim.x) {
    int y, w;
    split_index(i, g.Wp, y, w);
    uint32_t v;
    if (OP == 0) v = ~__ldg(a + i) & vmask(w, g.W);
    else if (OP == 1) v = __ldg(a + i) & __ldg(b + i);
    else if (OP == 2) v = __ldg(a + i) | __ldg(b + i);
    else if (OP == 3) v = 0u;
    else if (OP == 5) v = __ldg(a + i) & ~__ldg(b + i);
    else v = vmask(w, g.W);
    out[i] = v;
  }
}

__global__ void k_near(const uint32_t* __restrict__ a, MaskGeom g, int conn,
                       uint32_t* __restrict__ out) {
  const long long nwords = (long long)g.H * g.Wp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (long long)gridDim.x * blockDim.x) {
    int y, w;
    split_index(i, g.Wp, y, w);
    uint32_t r[3][3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int yy = y + dy - 1, ww = w + dx - 1;
        r[dy][dx] = (yy >= 0 && yy < g.H && ww >= 0 && ww < g.Wp)
                        ? __ldg(a + (size_t)yy * g.Wp + ww) : 0u;
      }
    out[i] = near_word(r[0][0], r[0][1], r[0][2], r[1][0], r[1][1], r[1][2], r[2][0],
                       r[2][1], r[2][2], conn) & vmask(w, g.W);
  }
}

// --------------------------------------------------------------- select --

__global__ void __launch_bounds__(EXEC_THREADS) k_select(const void* plane, int format, int pitch,
                                                         int H, int W, long long rank, float* out) {
  __shared__ SelectSmem s;
  float v = select_rank(s, plane, format, true, H, W, pitch, rank);
  if (threadIdx.x == 0) *out = v;
}

// Grid-wide radix select for large channels (a volume's 9 M voxels would
// keep the one-CTA select on a single SM for milliseconds): the same digits
// (8, 12, 12 bits of the order-preserving key), each pass one histogram
// kernel over the whole grid (shared-memory bins, then global atomics) and
// one warp that finds the digit holding the rank.
struct WideSel {
  uint32_t prefix, pmask;
  unsigned long long rank;
};

__global__ void k_sel_init(WideSel* st, long long rank) {
  st->prefix = 0;
  st->pmask = 0;
  st->rank = (unsigned long long)rank;
}

// Each thread takes SEL_UNR elements a grid stride apart per iteration (their
// loads in flight together); the row and column of an element are stepped
// by the stride instead of divided out.  A warp whose elements all fall in
// one bin (a background value) counts them with one shared atomic, else
// each element with its own; a warp none of whose elements passes the
// prefix skips both.
constexpr int SEL_UNR = 4;
__global__ void __launch_bounds__(256) k_sel_hist(const void* plane, int format, int pitch, int H,
                                                  int W, const WideSel* st, int sh, int nb,
                                                  uint32_t* hist) {
  __shared__ uint32_t h[4096];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t prefix = st->prefix, pmask = st->pmask;
  const int lane = threadIdx.x & 31;
  const long long n = (long long)H * W;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int sy = (int)(stride / W), sx = (int)(stride - (long long)sy * W);
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int y = (int)(i / W), x = (int)(i - (long long)y * W);
  // warp-uniform loop (every lane runs the ballots and the match)
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += SEL_UNR * stride) {
    uint32_t key[SEL_UNR];
    bool in[SEL_UNR];
#pragma unroll
    for (int u = 0; u < SEL_UNR; ++u) {
      in[u] = i < n;
      key[u] = in[u] ? f2key(ld_px(plane, format, true, (size_t)y * pitch + x)) : 0u;
      i += stride;
      y += sy;
      x += sx;
      if (x >= W) { x -= W; ++y; }
    }
#pragma unroll
    for (int u = 0; u < SEL_UNR; ++u) {
      const bool ok = in[u] && (key[u] & pmask) == prefix;
      if (!__any_sync(0xFFFFFFFFu, ok)) continue;
      const uint32_t bin = (key[u] >> sh) & (uint32_t)(nb - 1);
      int same = 0;
      __match_all_sync(0xFFFFFFFFu, ok ? bin : 0xFFFFFFFFu, &same);
      if (same) {  // the whole warp in one bin (a background value)
        if (lane == 0) atomicAdd(&h[bin], 32u);
      } else if (ok) {
        atomicAdd(&h[bin], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One warp: lane l sums bins [l * per, (l + 1) * per); a scan finds the lane
// whose bins hold the rank, which walks them.  The last pass writes the value.
__global__ void k_sel_pick(const uint32_t* hist, int sh, int nb, WideSel* st, float* out) {
  const int lane = threadIdx.x;
  const int per = nb / 32;
  unsigned long long sum = 0;
  for (int q = 0; q < per; ++q) sum += hist[lane * per + q];
  unsigned long long incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned long long rank = st->rank, excl = incl - sum;
  __syncwarp();
  if (sum > 0 && excl <= rank && rank < incl) {  // exactly one lane
    unsigned long long acc = excl;
    for (int q = 0; q < per; ++q) {
      const int b = lane * per + q;
      if (acc + hist[b] > rank) {
        st->prefix |= (uint32_t)b << sh;
        st->pmask |= (uint32_t)(nb - 1) << sh;
        st->rank = rank - acc;
        if (out) *out = key2f(st->prefix);
        break;
      }
      acc += hist[b];
    }
  }
}

// ----------------------------------------------------------- arithmetic --

// out = a (op) b pixel by pixel over H x W (row pitch `pitch` elements); b
// is a plane or, when null, the constant c.  One IEEE rounding per pixel.
__global__ void k_arith(int op, const void* __restrict__ a, int a_format, const void* b,
                        int b_format, float c, float* out, int H, int W, int pitch) {
  const long long n = (long long)H * W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int y, x;
    split_index(i, W, y, x);
    const size_t off = (size_t)y * pitch + x;
    const float u = ld_px(a, a_format, false, off);
    const float w = b ? ld_px(b, b_format, false, off) : c;
    float z;
    switch (op) {
      case A_ADD: z = __fadd_rn(u, w); break;
      case A_SUB: z = __fsub_rn(u, w); break;
      case A_MUL: z = __fmul_rn(u, w); break;
      default: z = __fdiv_rn(u, w); break;
    }
    out[off] = z;
  }
}

// ------------------------------------------------------------------ ccl --

__global__ void __launch_bounds__(EXEC_THREADS, 2)
k_ccl_local(const uint32_t* mask, const uint32_t* phi1, MaskGeom g, int tiles_x, int conn,
            CclScratch sc, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CclSmem& s = *reinterpret_cast<CclSmem*>(smem_raw);
  const CclGeom geo = ccl_geom(g.H, g.W, g.Wp, blockIdx.x, tiles_x, slice_rows(g), ccl_rows(g));
  const int npx = g.H * g.W;
  const bool labels = phi1 == nullptr;  // full labelling: canonical minimum pixel
  if (!ccl_tile_label(s, mask, phi1, geo, conn, labels, status)) return;
  ccl_encode_roots(s, geo, labels ? ENC_PUBLISH : ENC_PUBLISH_RZ, sc.G, labels ? npx : 2 * npx,
                   npx, status);
  ccl_publish_border(s, geo, sc.G);
  ccl_tile_save(s, sc.tpar + (size_t)blockIdx.x * sc.tile_cap,
                sc.tflag + (size_t)blockIdx.x * sc.tile_cap);
}

// glen: entries of G (H*W for labels, 2*H*W for rho keys).
__global__ void k_ccl_merge(const uint32_t* mask, MaskGeom g, int tiles_x, int conn, int32_t* G,
                            int glen, int32_t* status) {
  const int Hs = slice_rows(g);
  const int n = merge_units(g.H, g.Wp, tiles_x, Hs, ccl_rows(g));
  const int wpb = blockDim.x >> 5;
  for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < n; u += gridDim.x * wpb)
    ccl_merge_unit(mask, g.H, g.W, g.Wp, u, conn, G, glen, status, Hs, ccl_rows(g));
}

__global__ void __launch_bounds__(EXEC_THREADS, 2)
k_ccl_final_labels(const uint32_t* mask, MaskGeom g, int tiles_x, int conn, CclScratch sc,
                   int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CclSmem& s = *reinterpret_cast<CclSmem*>(smem_raw);
  const CclGeom geo = ccl_geom(g.H, g.W, g.Wp, blockIdx.x, tiles_x, slice_rows(g), ccl_rows(g));
  const int npx = g.H * g.W;
  if (!ccl_tile_load(s, mask, geo, conn, sc.tpar + (size_t)blockIdx.x * sc.tile_cap,
                     sc.tflag + (size_t)blockIdx.x * sc.tile_cap, status))
    return;
  ccl_encode_roots(s, geo, ENC_LABEL, sc.G, npx, npx, status);
  ccl_write_labels(s, geo, sc.G);
}

__global__ void __launch_bounds__(EXEC_THREADS, 2)
k_rz_final(const uint32_t* phi1, const uint32_t* phi2, MaskGeom g, int tiles_x, int conn,
           CclScratch sc, uint32_t* Z, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CclSmem& s = *reinterpret_cast<CclSmem*>(smem_raw);
  const CclGeom geo = ccl_geom(g.H, g.W, g.Wp, blockIdx.x, tiles_x, slice_rows(g), ccl_rows(g));
  const int npx = g.H * g.W;
  if (!ccl_tile_load(s, phi2, geo, conn, sc.tpar + (size_t)blockIdx.x * sc.tile_cap,
                     sc.tflag + (size_t)blockIdx.x * sc.tile_cap, status))
    return;
  ccl_encode_roots(s, geo, ENC_SELECT, sc.G, 2 * npx, npx, status);
  ccl_write_select(s, geo, Z);
}

// ----------------------------------------------------------- conversion --

__global__ void k_pack_u8(const uint8_t* __restrict__ src, MaskGeom g, uint32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long nwords = (long long)g.H * g.Wp;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nwords;
       i += nwarps) {
    int y, w;
    split_index(i, g.Wp, y, w);
    const int x = 32 * w + lane;
    const bool p = (x < g.W) && src[(size_t)y * g.W + x] != 0;
    const uint32_t word = __ballot_sync(FULL, p);
    if (lane == 0) out[i] = word;
  }
}

__global__ void k_unpack_u8(const uint32_t* __restrict__ src, MaskGeom g, uint8_t* __restrict__ out) {
  const long long n = (long long)g.H * g.W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int y, x;
    split_index(i, g.W, y, x);
    out[i] = (uint8_t)((__ldg(src + (size_t)y * g.Wp + (x >> 5)) >> (x & 31)) & 1u);
  }
}

__global__ void k_clear_padding(uint32_t* m, MaskGeom g) {
  const long long nwords = (long long)g.H * g.Wp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (long long)gridDim.x * blockDim.x) {
    int y, w;
    split_index(i, g.Wp, y, w);
    m[i] &= vmask(w, g.W);
  }
}

}  // namespace

// ============================================================ wrappers ==

cudaError_t launch_threshold(const void* plane, int format, int pitch, MaskGeom g, float t,
                             const float* t_dev, bool lt, uint32_t* out, cudaStream_t st) {
  long long nwords = (long long)g.H * g.Wp;
  k_threshold<<<grid_for(nwords * 4, kThreads * 4), kThreads, 0, st>>>(plane, format, pitch, g,
                                                                      t, t_dev, lt, out);
  return cudaGetLastError();
}

cudaError_t launch_not(const uint32_t* a, MaskGeom g, uint32_t* out, cudaStream_t st) {
  k_pointwise<0><<<grid_for((long long)g.H * g.Wp, kThreads * 4), kThreads, 0, st>>>(a, nullptr,
                                                                                    g, out);
  return cudaGetLastError();
}
cudaError_t launch_and(const uint32_t* a, const uint32_t* b, MaskGeom g, uint32_t* out,
                       cudaStream_t st) {
  k_pointwise<1><<<grid_for((long long)g.H * g.Wp, kThreads * 4), kThreads, 0, st>>>(a, b, g,
                                                                                    out);
  return cudaGetLastError();
}
cudaError_t launch_or(const uint32_t* a, const uint32_t* b, MaskGeom g, uint32_t* out,
                      cudaStream_t st) {
  k_pointwise<2><<<grid_for((long long)g.H * g.Wp, kThreads * 4), kThreads, 0, st>>>(a, b, g,
                                                                                    out);
  return cudaGetLastError();
}
cudaError_t launch_andnot(const uint32_t* a, const uint32_t* b, MaskGeom g, uint32_t* out,
                          cudaStream_t st) {
  k_pointwise<5><<<grid_for((long long)g.H * g.Wp, kThreads * 4), kThreads, 0, st>>>(a, b, g,
                                                                                    out);
  return cudaGetLastError();
}
cudaError_t launch_const(MaskGeom g, bool value, uint32_t* out, cudaStream_t st) {
  if (value)
    k_pointwise<4><<<grid_for((long long)g.H * g.Wp, kThreads * 4), kThreads, 0, st>>>(
        nullptr, nullptr, g, out);
  else
    k_pointwise<3><<<grid_for((long long)g.H * g.Wp, kThreads * 4), kThreads, 0, st>>>(
        nullptr, nullptr, g, out);
  return cudaGetLastError();
}
cudaError_t launch_near(const uint32_t* a, MaskGeom g, int conn, uint32_t* out,
                        cudaStream_t st) {
  k_near<<<grid_for((long long)g.H * g.Wp, kThreads * 2), kThreads, 0, st>>>(a, g, conn, out);
  return cudaGetLastError();
}
cudaError_t launch_select(const void* plane, int format, int pitch, int H, int W, long long rank,
                          float* out, cudaStream_t st) {
  k_select<<<1, EXEC_THREADS, 0, st>>>(plane, format, pitch, H, W, rank, out);
  return cudaGetLastError();
}

size_t select_wide_scratch_bytes() { return 4096 * sizeof(uint32_t) + 256; }

cudaError_t launch_select_wide(const void* plane, int format, int pitch, int H, int W,
                               long long rank, float* out, void* scratch, cudaStream_t st) {
  uint32_t* hist = static_cast<uint32_t*>(scratch);
  WideSel* ws = reinterpret_cast<WideSel*>(static_cast<char*>(scratch) + 4096 * sizeof(uint32_t));
  k_sel_init<<<1, 1, 0, st>>>(ws, rank);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  const int shifts[3] = {24, 12, 0}, widths[3] = {8, 12, 12};
  for (int pass = 0; pass < 3; ++pass) {
    const int nb = 1 << widths[pass];
    if ((e = cudaMemsetAsync(hist, 0, nb * sizeof(uint32_t), st))) return e;
    k_sel_hist<<<grid_for((long long)H * W, 256 * 8), 256, 0, st>>>(plane, format, pitch, H, W, ws,
                                                                   shifts[pass], nb, hist);
    if ((e = cudaGetLastError())) return e;
    k_sel_pick<<<1, 32, 0, st>>>(hist, shifts[pass], nb, ws, pass == 2 ? out : nullptr);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_arith(int op, const void* a, int a_format, const void* b, int b_format, float c,
                         float* out, int H, int W, int pitch, cudaStream_t st) {
  k_arith<<<grid_for((long long)H * W, kThreads), kThreads, 0, st>>>(op, a, a_format, b, b_format,
                                                                    c, out, H, W, pitch);
  return cudaGetLastError();
}

int ccl_tiles_y(int H, int Hs, int cth) {
  if (Hs <= 0) Hs = H;
  return (H / Hs) * ((Hs + cth - 1) / cth);
}
int ccl_tiles_x(int Wp) { return (Wp + CCL_TWW - 1) / CCL_TWW; }
size_t ccl_smem_bytes() { return sizeof(CclSmem); }

// The labelling kernels need more than 48 KB of dynamic shared memory; the
// attribute is set once per device (guarded: host threads may call the
// labelling entry points concurrently, on different devices).
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_attr_mu;
bool g_attr_done[kMaxDevices] = {};
}  // namespace

static cudaError_t ccl_set_attrs();
cudaError_t ccl_configure() { return ccl_set_attrs(); }

static cudaError_t ccl_set_attrs() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (g_attr_done[dev]) return cudaSuccess;
  const int sm = (int)sizeof(CclSmem);
  if ((e = cudaFuncSetAttribute(k_ccl_local, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_ccl_final_labels,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_rz_final, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
    return e;
  g_attr_done[dev] = true;
  return cudaSuccess;
}

long long ccl_merge_units(int H, int Wp, int Hs, int cth) {
  if (Hs <= 0) Hs = H;
  return (long long)(H / Hs) * ((Hs + cth - 1) / cth - 1) * Wp +
         (long long)(ccl_tiles_x(Wp) - 1) * ((H + 31) / 32);
}
int ccl_tile_cap_host(int Wp, int cth) { return (cth / 2) * std::min(CCL_TWW, Wp) * 32; }

cudaError_t launch_ccl_labels(const uint32_t* mask, MaskGeom g, int conn, CclScratch sc,
                              int32_t* status, cudaStream_t st) {
  cudaError_t e = ccl_set_attrs();
  if (e) return e;
  const int ty = ccl_tiles_y(g.H, g.Hs, ccl_rows(g)), tx = ccl_tiles_x(g.Wp);
  const size_t sm = sizeof(CclSmem);
  int32_t* labels = sc.G;
  k_ccl_local<<<ty * tx, EXEC_THREADS, sm, st>>>(mask, nullptr, g, tx, conn, sc, status);
  if ((e = cudaGetLastError())) return e;
  const long long nm = ccl_merge_units(g.H, g.Wp, g.Hs, ccl_rows(g)) * 32LL;
  if (nm > 0) {
    k_ccl_merge<<<grid_for(nm, kThreads), kThreads, 0, st>>>(mask, g, tx, conn, labels,
                                                             g.H * g.W, status);
    if ((e = cudaGetLastError())) return e;
  }
  k_ccl_final_labels<<<ty * tx, EXEC_THREADS, sm, st>>>(mask, g, tx, conn, sc, status);
  return cudaGetLastError();
}

cudaError_t launch_rz(const uint32_t* phi1, const uint32_t* phi2, MaskGeom g, int conn,
                      CclScratch sc, uint32_t* Z, int32_t* status, cudaStream_t st) {
  cudaError_t e = ccl_set_attrs();
  if (e) return e;
  const int ty = ccl_tiles_y(g.H, g.Hs, ccl_rows(g)), tx = ccl_tiles_x(g.Wp);
  const size_t sm = sizeof(CclSmem);
  k_ccl_local<<<ty * tx, EXEC_THREADS, sm, st>>>(phi2, phi1, g, tx, conn, sc, status);
  if ((e = cudaGetLastError())) return e;
  const long long nm = ccl_merge_units(g.H, g.Wp, g.Hs, ccl_rows(g)) * 32LL;
  if (nm > 0) {
    k_ccl_merge<<<grid_for(nm, kThreads), kThreads, 0, st>>>(phi2, g, tx, conn, sc.G,
                                                             2 * g.H * g.W, status);
    if ((e = cudaGetLastError())) return e;
  }
  k_rz_final<<<ty * tx, EXEC_THREADS, sm, st>>>(phi1, phi2, g, tx, conn, sc, Z, status);
  return cudaGetLastError();
}

cudaError_t launch_pack_u8(const uint8_t* src, MaskGeom g, uint32_t* out, cudaStream_t st) {
  k_pack_u8<<<grid_for((long long)g.H * g.Wp * 32, kThreads * 4), kThreads, 0, st>>>(src, g,
                                                                                    out);
  return cudaGetLastError();
}
cudaError_t launch_unpack_u8(const uint32_t* src, MaskGeom g, uint8_t* out, cudaStream_t st) {
  k_unpack_u8<<<grid_for((long long)g.H * g.W, kThreads * 8), kThreads, 0, st>>>(src, g, out);
  return cudaGetLastError();
}
cudaError_t launch_clear_padding(uint32_t* m, MaskGeom g, cudaStream_t st) {
  k_clear_padding<<<grid_for((long long)g.H * g.Wp, kThreads * 4), kThreads, 0, st>>>(m, g);
  return cudaGetLastError();
}

}  // namespace vl
