// Connected components on bit-packed masks, and the component select that
// reachability reduces to (Sec. 3.2: rho phi1[phi2] = N(phi1 or Z), Z the
// phi2-components that meet N phi1).
//
// Design (sm_103a, union-find, no host round trips -- unlike the paper's
// iterated pointer jumping with host-checked termination, Sec. 3.3):
//   1. tile-local: one CTA labels a tile of CCL_TH rows x CCL_TWW words.
//      Horizontal runs of foreground pixels are the union-find elements (run
//      starts come from bit tricks on the packed words); runs of adjacent
//      rows are united in shared memory with atomicMin.  Run ids follow the
//      raster order, so a local root is the run holding the minimum pixel.
//   2. publish: every foreground pixel on the tile border, and every local
//      root that reaches the border, gets an entry G[gid] in a global
//      union-find array indexed by linear pixel id gid = y*W + x.
//   3. merge: pixels adjacent across tile borders are united in G with
//      atomicMin (links always point to smaller gids, so no cycles).
//   4. final: each tile relabels again and resolves its border roots in G.
// Labels are canonical: the minimum linear index of each component.
#pragma once
#include "dev_common.cuh"

namespace vl {

constexpr uint32_t FULL = 0xFFFFFFFFu;

struct CclSmem {
  uint32_t m[CCL_TH][CCL_TWW];
  uint32_t st[CCL_TH][CCL_TWW];
  int32_t pre[CCL_TH][CCL_TWW];
  int32_t base[CCL_TH + 1];
  int32_t nruns;
  int32_t pad;
  int32_t parent[CCL_MAXRUNS];
  uint8_t flag[CCL_MAXRUNS];  // bit0 seed, bit1 on tile border, bit2 selected
};

struct CclGeom {
  int H, W, Wp;
  int r0, w0;   // tile origin: image row, image word
  int th, tww;  // rows and words of this tile
};

VL_DEV CclGeom ccl_geom(int H, int W, int Wp, int tile, int tiles_x) {
  CclGeom g;
  g.H = H; g.W = W; g.Wp = Wp;
  int ty = tile / tiles_x, tx = tile - ty * tiles_x;
  g.r0 = ty * CCL_TH;
  g.w0 = tx * CCL_TWW;
  g.th = min(CCL_TH, H - g.r0);
  g.tww = min(CCL_TWW, Wp - g.w0);
  return g;
}

VL_DEV int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// ---------------------------------------------------------- shared u-f --

VL_DEV int s_find(int32_t* par, int x, int cap) {
  volatile int32_t* p = par;
  for (int it = 0; it < cap; ++it) {
    int q = p[x];
    if (q == x) return x;
    int r = p[q];
    if (r != q) p[x] = r;  // path halving: r is an ancestor of x
    x = q;
  }
  return -1;
}

// Unite the sets of a and b; the smaller root wins.  Returns false if a
// bounded loop ran out (impossible unless memory is corrupted).
VL_DEV bool s_union(int32_t* par, int a, int b, int cap) {
  for (int it = 0; it < cap; ++it) {
    a = s_find(par, a, cap);
    b = s_find(par, b, cap);
    if (a < 0 || b < 0) return false;
    if (a == b) return true;
    if (a < b) { int t = a; a = b; b = t; }
    int old = atomicMin(&par[a], b);
    if (old == a) return true;
    a = old;
  }
  return false;
}

// ---------------------------------------------------------- global u-f --

// Root of x in G.  With `compress`, path halving rewrites G[x] to its
// grandparent (an ancestor, so the forest stays valid under concurrent
// unions).  The final relabelling pass must not compress: there, entries of
// finished tiles already hold their final labels.
VL_DEV int g_find(int32_t* G, int x, int cap, int32_t* status, bool compress = true) {
  for (int it = 0; it < cap; ++it) {
    int p = ldcg(&G[x]);
    if (p == x) return x;
    int r = ldcg(&G[p]);
    if (r == p) return p;
    if (compress) G[x] = r;
    x = r;
  }
  set_status(status, ST_INTERNAL);
  return x;
}

VL_DEV void g_union(int32_t* G, int a, int b, int cap, int32_t* status) {
  for (int it = 0; it < cap; ++it) {
    a = g_find(G, a, cap, status);
    b = g_find(G, b, cap, status);
    if (a == b) return;
    if (a < b) { int t = a; a = b; b = t; }
    int old = atomicMin(&G[a], b);
    if (old == a) return;
    a = old;
  }
  set_status(status, ST_INTERNAL);
}

// ------------------------------------------------------- tile labelling --

VL_DEV int run_id(const CclSmem& s, int row, int x) {
  int w = x >> 5;
  return s.base[row] + s.pre[row][w] + __popc(s.st[row][w] & le_mask(x & 31)) - 1;
}

VL_DEV bool bit_at(const CclSmem& s, int row, int x) {
  return (s.m[row][x >> 5] >> (x & 31)) & 1u;
}

// Leftmost foreground pixel of `row` among the pixels adjacent to column x
// (x-1..x+1 for 8-adjacency, x for 4), inside the tile; -1 if none.
VL_DEV int window_hit(const CclSmem& s, int row, int x, int width, int conn) {
  if (conn == 8 && x >= 1 && bit_at(s, row, x - 1)) return x - 1;
  if (bit_at(s, row, x)) return x;
  if (conn == 8 && x + 1 < width && bit_at(s, row, x + 1)) return x + 1;
  return -1;
}

// Dilation of mask `a` at (image row y, image word w) for one warp whose
// lanes hold consecutive words w0 + lane; lanes >= n are idle but take part
// in the shuffles.  Pixels outside the image are false.
VL_DEV uint32_t warp_near_row(const uint32_t* a, int H, int W, int Wp, int y,
                              int w0, int lane, int n, int conn) {
  int w = w0 + lane;
  bool in = lane < n;
  uint32_t u = 0, c = 0, d = 0;
  if (in) {
    if (y > 0) u = ldcg(&a[(size_t)(y - 1) * Wp + w]);
    c = ldcg(&a[(size_t)y * Wp + w]);
    if (y + 1 < H) d = ldcg(&a[(size_t)(y + 1) * Wp + w]);
  }
  uint32_t ul = __shfl_up_sync(FULL, u, 1), cl = __shfl_up_sync(FULL, c, 1),
           dl = __shfl_up_sync(FULL, d, 1);
  uint32_t ur = __shfl_down_sync(FULL, u, 1), cr = __shfl_down_sync(FULL, c, 1),
           dr = __shfl_down_sync(FULL, d, 1);
  if (in && lane == 0) {
    ul = cl = dl = 0;
    if (w > 0) {
      if (y > 0) ul = ldcg(&a[(size_t)(y - 1) * Wp + w - 1]);
      cl = ldcg(&a[(size_t)y * Wp + w - 1]);
      if (y + 1 < H) dl = ldcg(&a[(size_t)(y + 1) * Wp + w - 1]);
    }
  }
  if (in && lane == n - 1) {
    ur = cr = dr = 0;
    if (w + 1 < Wp) {
      if (y > 0) ur = ldcg(&a[(size_t)(y - 1) * Wp + w + 1]);
      cr = ldcg(&a[(size_t)y * Wp + w + 1]);
      if (y + 1 < H) dr = ldcg(&a[(size_t)(y + 1) * Wp + w + 1]);
    }
  }
  if (!in) return 0;
  return near_word(ul, u, ur, cl, c, cr, dl, d, dr, conn) & vmask(w, W);
}

// Label one tile in shared memory.  On return (after a block barrier):
// s.m/st/pre/base describe the runs, s.parent[i] is the local root of run i,
// s.flag[root] has bit0 set when a seed pixel lies in the component (if
// phi1 != nullptr: seed = mask and N phi1), bit1 when the component reaches
// the tile border.  Must be called by every thread of the block.
VL_DEV void ccl_tile_label(CclSmem& s, const uint32_t* mask, const uint32_t* phi1,
                           const CclGeom& g, int conn, int32_t* status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  // 1. load, run starts, per-row prefix of run counts
  for (int r = warp; r < g.th; r += nw) {
    uint32_t m = 0;
    if (lane < g.tww) m = ldcg(&mask[(size_t)(g.r0 + r) * g.Wp + g.w0 + lane]);
    uint32_t left = __shfl_up_sync(FULL, m, 1);
    if (lane == 0) left = 0;
    uint32_t st = m & ~((m << 1) | (left >> 31));
    int c = __popc(st);
    int incl = warp_incl_scan(c, lane);
    s.m[r][lane] = m;
    s.st[r][lane] = st;
    s.pre[r][lane] = incl - c;
    if (lane == 31) s.base[r + 1] = incl;
  }
  __syncthreads();
  if (warp == 0) {
    int v = (lane < g.th) ? s.base[lane + 1] : 0;
    int incl = warp_incl_scan(v, lane);
    __syncwarp();
    if (lane < g.th) s.base[lane] = incl - v;
    if (lane == 31) { s.base[g.th] = incl; s.nruns = incl; }
  }
  __syncthreads();
  const int nruns = s.nruns;
  for (int i = threadIdx.x; i < nruns; i += blockDim.x) {
    s.parent[i] = i;
    s.flag[i] = 0;
  }
  __syncthreads();
  // 2. unite runs of adjacent rows: each run start looks at the window of
  // the other row; the leftmost hit is enough (every overlapping pair of
  // runs is met at the start of one of them).
  const int width = 32 * g.tww;
  const int cap = nruns + 64;
  bool ok = true;
  for (int r = 1 + warp; r < g.th; r += nw) {
    if (lane < g.tww) {
      uint32_t sc = s.st[r][lane];
      while (sc) {
        int b = __ffs(sc) - 1;
        sc &= sc - 1;
        int x = 32 * lane + b;
        int p = window_hit(s, r - 1, x, width, conn);
        if (p >= 0) ok &= s_union(s.parent, run_id(s, r, x), run_id(s, r - 1, p), cap);
      }
      uint32_t su = s.st[r - 1][lane];
      while (su) {
        int b = __ffs(su) - 1;
        su &= su - 1;
        int x = 32 * lane + b;
        int p = window_hit(s, r, x, width, conn);
        if (p >= 0) ok &= s_union(s.parent, run_id(s, r - 1, x), run_id(s, r, p), cap);
      }
    }
  }
  __syncthreads();
  // 3. flatten
  for (int i = threadIdx.x; i < nruns; i += blockDim.x) {
    int root = s_find(s.parent, i, cap);
    if (root < 0) { ok = false; root = i; }
    s.parent[i] = root;
  }
  if (!ok) set_status(status, ST_INTERNAL);
  __syncthreads();
  // 4. seeds: components holding a pixel of mask and N phi1
  if (phi1 != nullptr) {
    for (int r = warp; r < g.th; r += nw) {
      uint32_t z = warp_near_row(phi1, g.H, g.W, g.Wp, g.r0 + r, g.w0, lane, g.tww, conn);
      uint32_t m = s.m[r][lane];
      z &= m;
      uint32_t zl = __shfl_up_sync(FULL, z, 1);
      if (lane == 0) zl = 0;
      uint32_t zs = z & ~((z << 1) | (zl >> 31));
      while (zs) {
        int b = __ffs(zs) - 1;
        zs &= zs - 1;
        s.flag[s.parent[run_id(s, r, 32 * lane + b)]] = 1;
      }
    }
    __syncthreads();
  }
  // 5. components on the tile border
  for (int r = warp; r < g.th; r += nw) {
    if (lane < g.tww) {
      uint32_t m = s.m[r][lane];
      if (r == 0 || r == g.th - 1) {
        uint32_t sc = s.st[r][lane];
        while (sc) {
          int b = __ffs(sc) - 1;
          sc &= sc - 1;
          int root = s.parent[run_id(s, r, 32 * lane + b)];
          s.flag[root] |= 2;
        }
      }
      if (lane == 0 && (m & 1u)) s.flag[s.parent[s.base[r]]] |= 2;
      if (lane == g.tww - 1 && (m >> 31)) s.flag[s.parent[s.base[r + 1] - 1]] |= 2;
    }
  }
  __syncthreads();
}

// Root of run rid after roots have been encoded (parent[root] < 0).
VL_DEV int root_of(const CclSmem& s, int rid) {
  int p = s.parent[rid];
  return p >= 0 ? p : rid;
}
// Encoded value of the root of run rid (see ccl_encode_roots).
VL_DEV int root_value(const CclSmem& s, int rid) {
  int p = s.parent[rid];
  if (p >= 0) p = s.parent[p];
  return -p - 2;
}

// Modes of ccl_encode_roots.
constexpr int ENC_PUBLISH = 0;  // value = root gid; publish border roots
constexpr int ENC_LABEL = 1;    // value = global label (border roots resolved in G)
constexpr int ENC_SELECT = 2;   // flag bit2 = component selected (rho); value = gid

// Visit every local root once (at its start pixel) and replace parent[root]
// by -(value + 2).  Block barrier at the end.
VL_DEV void ccl_encode_roots(CclSmem& s, const CclGeom& g, int mode, int32_t* G,
                             uint8_t* F, int32_t* flist, int32_t* fcount,
                             int flist_cap, int cap, int32_t* status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int r = warp; r < g.th; r += nw) {
    if (lane >= g.tww) continue;
    uint32_t sc = s.st[r][lane];
    while (sc) {
      int b = __ffs(sc) - 1;
      sc &= sc - 1;
      int x = 32 * lane + b;
      int rid = run_id(s, r, x);
      if (s.parent[rid] != rid) continue;
      int gid = (g.r0 + r) * g.W + 32 * g.w0 + x;
      uint8_t fl = s.flag[rid];
      int value = gid;
      if (mode == ENC_PUBLISH) {
        if (fl & 2) {
          G[gid] = gid;
          if (F) {
            F[gid] = fl & 1;
            if (fl & 1) {
              int k = atomicAdd(fcount, 1);
              if (k < flist_cap) flist[k] = gid;
              else set_status(status, ST_INTERNAL);
            }
          }
        }
      } else if (mode == ENC_LABEL) {
        if (fl & 2) value = g_find(G, gid, cap, status, false);
      } else {  // ENC_SELECT
        uint8_t sel = fl & 1;
        if (fl & 2) sel = ldcg(&F[g_find(G, gid, cap, status, false)]);
        if (sel) s.flag[rid] = fl | 4;
      }
      s.parent[rid] = -(value + 2);
    }
  }
  __syncthreads();
}

// Border pixels of the tile point at their local root's gid in G.
VL_DEV void ccl_publish_border(CclSmem& s, const CclGeom& g, int32_t* G) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int width = 32 * g.tww;
  for (int r = warp; r < g.th; r += nw) {
    const int y = g.r0 + r;
    if (r == 0 || r == g.th - 1) {
      for (int x = lane; x < width; x += 32)
        if (bit_at(s, r, x)) G[y * g.W + 32 * g.w0 + x] = root_value(s, run_id(s, r, x));
    } else if (lane == 0) {
      if (bit_at(s, r, 0)) G[y * g.W + 32 * g.w0] = root_value(s, s.base[r]);
      int xr = width - 1;
      if (bit_at(s, r, xr)) G[y * g.W + 32 * g.w0 + xr] = root_value(s, s.base[r + 1] - 1);
    }
  }
}

// Write labels of the tile (after ENC_LABEL): coalesced row segments.
VL_DEV void ccl_write_labels(const CclSmem& s, const CclGeom& g, int32_t* labels) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int x_end = min(32 * g.tww, g.W - 32 * g.w0);
  for (int r = warp; r < g.th; r += nw) {
    int32_t* row = labels + (size_t)(g.r0 + r) * g.W + 32 * g.w0;
    for (int x = lane; x < x_end; x += 32)
      row[x] = bit_at(s, r, x) ? root_value(s, run_id(s, r, x)) : -1;
  }
}

// Write Z = the selected components of the tile (after ENC_SELECT).
VL_DEV void ccl_write_select(const CclSmem& s, const CclGeom& g, uint32_t* Z) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int r = warp; r < g.th; r += nw) {
    if (lane >= g.tww) continue;
    uint32_t m = s.m[r][lane], st = s.st[r][lane];
    uint32_t f = 0, sc = st;
    while (sc) {
      int b = __ffs(sc) - 1;
      sc &= sc - 1;
      if (s.flag[root_of(s, run_id(s, r, 32 * lane + b))] & 4) f |= 1u << b;
    }
    if ((m & 1u) && !(st & 1u) && (s.flag[root_of(s, run_id(s, r, 32 * lane))] & 4)) f |= 1u;
    // a carry entering at the first pixel of a run clears the run and sets
    // the pixel after it, so ((m + f) ^ m) & m is exactly the selected runs
    uint32_t z = ((m + f) ^ m) & m;
    Z[(size_t)(g.r0 + r) * g.Wp + g.w0 + lane] = z;
  }
}

// --------------------------------------------------------- border merge --
// Work items of the merge: one per word of each horizontal tile border, one
// per row of each vertical tile border.
VL_DEV int merge_items(int H, int Wp, int tiles_y, int tiles_x) {
  return (tiles_y - 1) * Wp + (tiles_x - 1) * H;
}

VL_DEV uint32_t bitw(const uint32_t* m, int Wp, int y, int x) {
  return (ldcg(&m[(size_t)y * Wp + (x >> 5)]) >> (x & 31)) & 1u;
}

// Leftmost foreground pixel of row y among the columns adjacent to x.
VL_DEV int g_window_hit(const uint32_t* m, int W, int Wp, int y, int x, int conn) {
  if (conn == 8 && x >= 1 && bitw(m, Wp, y, x - 1)) return x - 1;
  if (bitw(m, Wp, y, x)) return x;
  if (conn == 8 && x + 1 < W && bitw(m, Wp, y, x + 1)) return x + 1;
  return -1;
}

VL_DEV void ccl_merge_item(const uint32_t* m, int H, int W, int Wp, int tiles_y,
                           int item, int conn, int32_t* G, int cap, int32_t* status) {
  const int nh = (tiles_y - 1) * Wp;
  if (item < nh) {
    int k = item / Wp + 1, w = item - (k - 1) * Wp;
    int yd = k * CCL_TH, yu = yd - 1;
    uint32_t md = ldcg(&m[(size_t)yd * Wp + w]), mu = ldcg(&m[(size_t)yu * Wp + w]);
    uint32_t mdl = w > 0 ? ldcg(&m[(size_t)yd * Wp + w - 1]) : 0u;
    uint32_t mul = w > 0 ? ldcg(&m[(size_t)yu * Wp + w - 1]) : 0u;
    uint32_t sd = md & ~((md << 1) | (mdl >> 31));
    uint32_t su = mu & ~((mu << 1) | (mul >> 31));
    while (sd) {
      int b = __ffs(sd) - 1;
      sd &= sd - 1;
      int x = 32 * w + b;
      int p = g_window_hit(m, W, Wp, yu, x, conn);
      if (p >= 0) g_union(G, yd * W + x, yu * W + p, cap, status);
    }
    while (su) {
      int b = __ffs(su) - 1;
      su &= su - 1;
      int x = 32 * w + b;
      int p = g_window_hit(m, W, Wp, yd, x, conn);
      if (p >= 0) g_union(G, yu * W + x, yd * W + p, cap, status);
    }
  } else {
    int j = item - nh;
    int k = j / H + 1, y = j - (k - 1) * H;
    int x0 = k * CCL_TWW * 32;
    if (x0 >= W) return;
    if (!bitw(m, Wp, y, x0 - 1)) return;
    int a = y * W + x0 - 1;
    if (bitw(m, Wp, y, x0)) g_union(G, a, y * W + x0, cap, status);
    if (conn == 8) {
      if (y > 0 && bitw(m, Wp, y - 1, x0)) g_union(G, a, (y - 1) * W + x0, cap, status);
      if (y + 1 < H && bitw(m, Wp, y + 1, x0)) g_union(G, a, (y + 1) * W + x0, cap, status);
    }
  }
}

}  // namespace vl
