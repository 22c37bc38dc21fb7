// Volumes: the logic of Sec. 2 on D x H x W voxel grids, the paper's outlook
// beyond 2D slices (Sec. 1 and Sec. 5).  A volume is stored as its D slices
// stacked into one image of D * H rows (slice z is rows [z * H, (z + 1) * H)),
// bit-packed like any mask, so thresholds, not/and and percentiles run the
// 2D kernels unchanged.  Only the operators that look at neighbours differ:
//   N   -- 26-adjacency: the 3 x 3 x 3 cube, i.e. the 2D 3 x 3 dilation of the
//          OR of the rows y-1..y+1 of slices z-1..z+1; 6-adjacency: the faces,
//          i.e. the 2D cross of slice z OR the same word of slices z-1, z+1.
//          Both clip at the volume's border (no voxels outside it).
//   CCL -- 2D labelling of every slice (tiles never straddle slices; the
//          in-slice adjacency is 8 for 26 and 4 for 6), then a merge between
//          neighbouring slices: the rows (z, y) and (z + 1, y + dy) with
//          dy in {-1, 0, 1} under a 3-voxel window (26), or (z, y) and
//          (z + 1, y) voxel on voxel (6); then every voxel takes its root.
//          Labels are canonical: the minimum linear index z*H*W + y*W + x.
//   rho -- as for images (Sec. 3.2): rho phi1[phi2] = N(phi1 or Z), Z the
//          phi2-components that meet N phi1; Z from the full labels of phi2,
//          a flag per component root set from the seed voxels.
#include "dev_ccl.cuh"
#include "dev_common.cuh"
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

// Word w of row `row` of the stored image, 0 outside [0, Wp).
VL_DEV uint32_t word_at(const uint32_t* a, int Wp, int row, int w) {
  return (w >= 0 && w < Wp) ? __ldg(a + (size_t)row * Wp + w) : 0u;
}

// out = N a, or (N a) and `with` when `with` is given.
__global__ void k_near3(const uint32_t* __restrict__ a, MaskGeom g, int conn,
                        const uint32_t* __restrict__ with, uint32_t* __restrict__ out) {
  const int Hs = slice_rows(g), D = g.H / Hs;
  const long long nwords = (long long)g.H * g.Wp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (long long)gridDim.x * blockDim.x) {
    int y, w;
    split_index(i, g.Wp, y, w);
    const int z = y / Hs, yz = y - z * Hs;
    uint32_t res;
    if (conn == 26) {
      uint32_t l = 0, c = 0, r = 0;  // OR of the 9 rows around, per column word
      for (int dz = -1; dz <= 1; ++dz) {
        const int zz = z + dz;
        if (zz < 0 || zz >= D) continue;
        for (int dy = -1; dy <= 1; ++dy) {
          const int yy = yz + dy;
          if (yy < 0 || yy >= Hs) continue;
          const int row = zz * Hs + yy;
          l |= word_at(a, g.Wp, row, w - 1);
          c |= word_at(a, g.Wp, row, w);
          r |= word_at(a, g.Wp, row, w + 1);
        }
      }
      res = hdil(l, c, r);
    } else {
      res = hdil(word_at(a, g.Wp, y, w - 1), word_at(a, g.Wp, y, w), word_at(a, g.Wp, y, w + 1));
      if (yz > 0) res |= word_at(a, g.Wp, y - 1, w);
      if (yz + 1 < Hs) res |= word_at(a, g.Wp, y + 1, w);
      if (z > 0) res |= word_at(a, g.Wp, y - Hs, w);
      if (z + 1 < D) res |= word_at(a, g.Wp, y + Hs, w);
    }
    res &= vmask(w, g.W);
    if (with) res &= __ldg(with + i);
    out[i] = res;
  }
}

// Unite the components of slices z and z + 1: one warp per row pair (z, y)
// -- placed by a 32-bit division -- looping over the row's words and, for
// 26-adjacency, the rows y - 1, y, y + 1 of slice z + 1.
// L holds, for every voxel of the mask, its component's key (after the 2D
// pass: the minimum index of its slice component, which is a root).
__global__ void k_zmerge(const uint32_t* m, MaskGeom g, int conn, int32_t* L, int32_t* status) {
  const int Hs = slice_rows(g), D = g.H / Hs;
  const int nd = conn == 26 ? 3 : 1;
  const long long rows = (long long)(D - 1) * Hs;
  const int npx = g.H * g.W;
  const long long wpb = blockDim.x >> 5;
  for (long long r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += gridDim.x * wpb) {
    int z, yz;  // uniform across the warp
    split_index(r, Hs, z, yz);
    for (int w = 0; w < g.Wp; ++w)
      for (int k = 0; k < nd; ++k) {
        const int yb = yz + (nd == 3 ? k - 1 : 0);
        if (yb < 0 || yb >= Hs) continue;
        ccl_merge_rows(m, g.W, g.Wp, z * Hs + yz, (z + 1) * Hs + yb, w, conn == 26 ? 8 : 4, L,
                       npx, status);
      }
  }
}

// Every voxel of the mask takes the root of its key (finds compress: a
// node only moves to an ancestor, and the root is the label of every node
// on the way).
__global__ void k_relabel(const uint32_t* m, MaskGeom g, int32_t* L, int32_t* status) {
  const int npx = g.H * g.W;
  // grid-stride over the voxels, row and column stepped instead of divided
  const int stride = gridDim.x * blockDim.x;
  const int sy = stride / g.W, sx = stride - sy * g.W;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int y, x;
  split_index(i, g.W, y, x);
  for (; i < npx; i += stride) {
    if ((__ldg(m + (size_t)y * g.Wp + (x >> 5)) >> (x & 31)) & 1u)
      L[i] = g_find(L, ldcg(&L[i]), npx, status);
    y += sy;
    x += sx;
    if (x >= g.W) { x -= g.W; ++y; }
  }
}

// F[label] = 1 for every seed voxel (benign races: every writer writes 1).
// Seeds lie in phi2, so the voxels of a run of seeds in a row share one
// component: only the first voxel of every run is looked up.
__global__ void k_seed_flags(const uint32_t* seed, MaskGeom g, const int32_t* L, uint8_t* F) {
  const long long nwords = (long long)g.H * g.Wp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (long long)gridDim.x * blockDim.x) {
    int y, w;
    split_index(i, g.Wp, y, w);
    const uint32_t cur = __ldg(seed + i) & vmask(w, g.W);
    const uint32_t prev = w > 0 ? __ldg(seed + i - 1) : 0u;
    uint32_t bits = cur & ~((cur << 1) | (prev >> 31));
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const int lab = __ldg(L + (size_t)y * g.W + 32 * w + b);
      if ((unsigned)lab < (unsigned)(g.H * g.W)) F[lab] = 1;
    }
  }
}

// Z = the voxels of phi2 whose component is flagged: one lookup per run of
// phi2 inside the word (a run is one component), the run's bits taken whole.
__global__ void k_select_flagged(const uint32_t* phi2, MaskGeom g, const int32_t* L,
                                 const uint8_t* F, uint32_t* Z) {
  const long long nwords = (long long)g.H * g.Wp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (long long)gridDim.x * blockDim.x) {
    int y, w;
    split_index(i, g.Wp, y, w);
    const uint32_t bits = __ldg(phi2 + i) & vmask(w, g.W);
    uint32_t starts = bits & ~(bits << 1), sel = 0;  // run starts inside this word
    while (starts) {
      const int b = __ffs(starts) - 1;
      starts &= starts - 1;
      // the run: bits b.. up to the first clear bit
      const uint32_t from = bits >> b;
      const uint32_t len_mask = ~from ? ((~from & (0u - ~from)) - 1u) : 0xFFFFFFFFu;
      const int lab = __ldg(L + (size_t)y * g.W + 32 * w + b);
      if ((unsigned)lab < (unsigned)(g.H * g.W) && F[lab]) sel |= len_mask << b;
    }
    Z[i] = sel;
  }
}

}  // namespace

cudaError_t launch_near3(const uint32_t* a, MaskGeom g, int conn, uint32_t* out, cudaStream_t st) {
  k_near3<<<grid_for((long long)g.H * g.Wp, kThreads * 2), kThreads, 0, st>>>(a, g, conn, nullptr,
                                                                            out);
  return cudaGetLastError();
}

cudaError_t launch_labels3(const uint32_t* mask, MaskGeom g, int conn, CclScratch sc,
                           int32_t* status, cudaStream_t st) {
  cudaError_t e = launch_ccl_labels(mask, g, conn == 26 ? 8 : 4, sc, status, st);
  if (e) return e;
  const int Hs = slice_rows(g), D = g.H / Hs;
  if (D < 2) return cudaSuccess;
  const long long rows = (long long)(D - 1) * Hs;  // one warp per row pair
  k_zmerge<<<grid_for(rows * 32, kThreads), kThreads, 0, st>>>(mask, g, conn, sc.G, status);
  if ((e = cudaGetLastError())) return e;
  k_relabel<<<grid_for((long long)g.H * g.W, kThreads * 4), kThreads, 0, st>>>(mask, g, sc.G, status);
  return cudaGetLastError();
}

cudaError_t launch_rz3(const uint32_t* phi1, const uint32_t* phi2, MaskGeom g, int conn,
                       Rz3Scratch sc, uint32_t* Z, int32_t* status, cudaStream_t st) {
  cudaError_t e = launch_labels3(phi2, g, conn, sc.ccl, status, st);
  if (e) return e;
  // seeds: the voxels of phi2 in N phi1
  k_near3<<<grid_for((long long)g.H * g.Wp, kThreads * 2), kThreads, 0, st>>>(phi1, g, conn, phi2,
                                                                            sc.seed);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemsetAsync(sc.F, 0, (size_t)g.H * g.W, st))) return e;
  const long long nwords = (long long)g.H * g.Wp;
  k_seed_flags<<<grid_for(nwords, kThreads * 2), kThreads, 0, st>>>(sc.seed, g, sc.ccl.G, sc.F);
  if ((e = cudaGetLastError())) return e;
  k_select_flagged<<<grid_for(nwords, kThreads * 2), kThreads, 0, st>>>(phi2, g, sc.ccl.G, sc.F, Z);
  return cudaGetLastError();
}

}  // namespace vl
