// Connected components on bit-packed masks, and the component select that
// reachability reduces to (Sec. 3.2: rho phi1[phi2] = N(phi1 or Z), Z the
// phi2-components that meet N phi1).
//
// Design (sm_103a, union-find, no host round trips -- unlike the paper's
// iterated pointer jumping with host-checked termination, Sec. 3.3):
//   1. tile-local: one CTA labels a tile of CCL_TH rows x CCL_TWW words.
//      The union-find elements are the connected pieces of two-row strips,
//      found with bit operations on the packed words; strips are united in
//      shared memory with atomicMin along a binary tree of strip boundaries.
//   2. publish: every foreground pixel on the tile border, and every local
//      root that reaches the border, gets an entry G[gid] in a global
//      union-find array indexed by linear pixel id gid = y*W + x.
//   3. merge: pixels adjacent across tile borders are united in G; a root
//      is linked under the smaller root by compare-and-swap, so only a node
//      that is still a root is ever re-pointed and links always point to
//      smaller gids (no cycles).
//   4. final: each tile relabels again and resolves its border roots in G.
// Labels are canonical: the minimum linear index of each component.
#pragma once
#include <climits>

#include "dev_common.cuh"

namespace vl {

constexpr uint32_t FULL = 0xFFFFFFFFu;

struct CclSmem {
  uint32_t m[CCL_TH][CCL_TWW];   // rows of the tile
  uint32_t u[CCL_NS][CCL_TWW];   // strip unions (row 2k | row 2k+1)
  uint32_t st[CCL_NS][CCL_TWW];  // strip-run starts
  int32_t pre[CCL_NS][CCL_TWW];  // starts before each word, per strip
  int32_t qc[CCL_NS][CCL_TWW];   // boundary anchor entering each word
  int32_t base[CCL_NS + 1];      // first strip-run id of each strip
  int32_t nruns;
  int32_t pad;
  int32_t parent[CCL_MAXRUNS];   // union-find; after labelling a root holds -(value + 2)
  uint8_t flag[CCL_MAXRUNS];     // bit0 seed, bit1 on tile border, bit2 selected
};

struct CclGeom {
  int H, W, Wp;
  int r0, w0;   // tile origin: image row, image word
  int th, tww;  // rows and words of this tile
};

// Tile `tile` of an image of H rows, or of a volume stored as its slices of
// Hs rows stacked (H = depth * Hs; Hs = H for an image): tiles never
// straddle two slices, so the tile-local labelling stays inside one slice.
// cth: rows of a tile (an even number up to CCL_TH; smaller tiles give small
// images more tiles to spread over the GPU).
VL_DEV CclGeom ccl_geom(int H, int W, int Wp, int tile, int tiles_x, int Hs, int cth = CCL_TH) {
  CclGeom g;
  g.H = H; g.W = W; g.Wp = Wp;
  const int tys = (Hs + cth - 1) / cth;  // tile rows per slice
  const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
  const int z = ty / tys, tyz = ty - z * tys;
  g.r0 = z * Hs + tyz * cth;
  g.w0 = tx * CCL_TWW;
  g.th = min(cth, Hs - tyz * cth);
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

// cap = strip runs + 64: an index outside the runs, or a walk longer than
// cap, returns -1 (the caller reports RS_SUNION) instead of reading past
// the array.
VL_DEV int s_find(int32_t* par, int x, int cap) {
  volatile int32_t* p = par;
  if ((unsigned)x >= (unsigned)(cap - 64)) return -1;
  for (int it = 0; it < cap; ++it) {
    int q = p[x];
    if (q == x) return x;
    int r = p[q];
    if (r != q) p[x] = r;  // path halving: r is an ancestor of x
    x = q;
  }
  return -1;
}

// Roots of a and b, both chains walked side by side with path halving (each
// node passed is pointed at its grandparent, and the walk jumps there): on
// return a == b when the walks met (the same set; not necessarily a root),
// else both are roots.  False if an index is out of range or a bounded loop
// ran out (impossible unless memory is corrupted).
VL_DEV bool s_find2(int32_t* par, int& a, int& b, int cap) {
  volatile int32_t* p = par;
  const unsigned lim = (unsigned)(cap - 64);
  for (int it = 0; it < cap; ++it) {
    if (a == b) return true;
    if ((unsigned)a >= lim || (unsigned)b >= lim) return false;
    const int qa = p[a], qb = p[b];
    const bool ra = qa == a, rb = qb == b;
    if (ra && rb) return true;
    if ((unsigned)qa >= lim || (unsigned)qb >= lim) return false;
    const int ga = ra ? qa : p[qa], gb = rb ? qb : p[qb];
    if (!ra) {
      if (ga != qa) p[a] = ga;
      a = ga;
    }
    if (!rb) {
      if (gb != qb) p[b] = gb;
      b = gb;
    }
  }
  return false;
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

// Root of x in G.  With `compress`, every node on the path from x gets the
// root as its parent.  This is safe because a node's parent only ever moves
// to one of its ancestors: g_union links a node only while it is a root
// (compare-and-swap), and nodes on the path from x, and the root found, all
// lie on x's single chain of ancestors, the root above them (ids decrease
// along the chain).  In the final labelling pass G is the label array and
// finished tiles have written their labels into it: the label of every
// node on a path is the root the path ends at, the value a compression
// writes there too.
// npx: entries of G.  An entry outside [0, npx) can only come from
// corrupted state; it is reported (reason RS_GRANGE) and the walk stops at
// the last valid node instead of reading out of bounds.
VL_DEV int g_find(int32_t* G, int x, int npx, int32_t* status, bool compress = true) {
  const int cap = min(npx + 64, 1 << 22);
  if ((unsigned)x >= (unsigned)npx) {
    set_status(status, ST_INTERNAL | RS_GRANGE);
    return 0;
  }
  int root = x;
  int it = 0;
  for (; it < cap; ++it) {
    const int p = ldcg(&G[root]);
    if (p == root) break;
    if ((unsigned)p >= (unsigned)npx) {
      set_status(status, ST_INTERNAL | RS_GRANGE);
      return root;
    }
    root = p;
  }
  if (it == cap) {
    set_status(status, ST_INTERNAL | RS_GFIND);
    return root;
  }
  if (compress) {
    for (int k = 0; k < it && x > root; ++k) {
      const int p = ldcg(&G[x]);
      if (p <= root) break;
      G[x] = root;
      x = p;
    }
  }
  return root;
}

// Roots of a and b in G, both chains walked side by side, with path halving:
// each node passed is pointed at its grandparent.  Like the compression in
// g_find this only ever moves a node to one of its ancestors, and it costs no
// second walk.  On return a == b (same set; they need not be roots) or both
// are roots.  Only while the union-find is being built: in the final pass a
// node of a finished tile holds its final label, which a halving write would
// replace by an inner node.
VL_DEV void g_find2(int32_t* G, int& a, int& b, int npx, int32_t* status) {
  const int cap = min(npx + 64, 1 << 22);
  for (int it = 0; it < cap; ++it) {
    if (a == b) return;
    if ((unsigned)a >= (unsigned)npx || (unsigned)b >= (unsigned)npx) {
      set_status(status, ST_INTERNAL | RS_GRANGE);
      a = b = 0;
      return;
    }
    const int pa = ldcg(&G[a]), pb = ldcg(&G[b]);
    const bool ra = pa == a, rb = pb == b;
    if (ra && rb) return;
    if ((unsigned)pa >= (unsigned)npx || (unsigned)pb >= (unsigned)npx) {
      set_status(status, ST_INTERNAL | RS_GRANGE);
      a = b = 0;
      return;
    }
    const int ga = ra ? pa : ldcg(&G[pa]), gb = rb ? pb : ldcg(&G[pb]);
    if (!ra) {
      if (ga != pa) G[a] = ga;
      a = ga;
    }
    if (!rb) {
      if (gb != pb) G[b] = gb;
      b = gb;
    }
  }
  set_status(status, ST_INTERNAL | RS_GFIND);
  a = b = 0;
}

// Unite the sets of a and b: the larger root is linked under the smaller,
// by compare-and-swap so that only a node that is still a root is ever
// re-pointed.  (An atomicMin on a root that was linked meanwhile would move
// its whole tree to the other set for a moment; a concurrent compression
// following that fresh link could then carry a node of the other set into
// this one and strand the rest of that set.)  A failed swap retries from
// fresh roots.
VL_DEV void g_union(int32_t* G, int a, int b, int npx, int32_t* status) {
  const int cap = min(npx + 64, 1 << 22);
  for (int it = 0; it < cap; ++it) {
    g_find2(G, a, b, npx, status);
    if (a == b) return;
    if (a < b) { int t = a; a = b; b = t; }
    if (atomicCAS(&G[a], a, b) == a) return;
  }
  set_status(status, ST_INTERNAL | RS_GUNION);
}

// ------------------------------------------------------- tile labelling --
//
// Level 0 is bit-parallel: in a strip of two rows A (top) and B, the
// components under 8-adjacency are exactly the runs of A | B (consecutive
// set columns always touch, diagonally at least); under 4-adjacency they are
// those runs cut where the set row switches from A-only to B-only (or back)
// between two columns.  These "strip runs" are the union-find elements.
// Strips are then merged across the CCL_NS - 1 strip boundaries in a
// binary-tree order (boundary b at level = trailing ones of b, plus one), so
// every level unites disjoint groups of strips and the trees stay shallow.
// Across a boundary (rows A' = last row of the upper strip, B' = first row of
// the lower one), the same two-row rule holds: every set pixel of A' and B'
// inside one run of A' | B' (cut the same way for 4-adjacency) is connected,
// so each row run starting inside it is united with the run's anchor.

// The lowest bit of x in every segment of a 32-bit word, segments starting
// at bit 0 and at every set bit of s: clear the bits of x that have another
// bit of x below them in the same segment.  "Has an x bit below in its
// segment" is the carry into that position of P + x, P = ~s | x: a carry
// starts at every x bit, runs on through positions not in s, and dies at
// a bit of s that is not in x.
VL_DEV uint32_t first_in_segments(uint32_t x, uint32_t s) {
  const uint32_t p = ~s | x;
  const uint32_t carry_in = (p + x) ^ p ^ x;
  return x & ~(carry_in & ~s);
}

// Strip-run starts of a two-row strip (a, b) given the previous word's
// (a, b) (0 at the tile's left edge).
VL_DEV uint32_t strip_starts(uint32_t a, uint32_t b, uint32_t al, uint32_t bl, int conn) {
  const uint32_t u = a | b, ul = al | bl;
  uint32_t st = u & ~((u << 1) | (ul >> 31));
  if (conn == 4) {
    const uint32_t ao = a & ~b, bo = b & ~a, aol = al & ~bl, bol = bl & ~al;
    st |= (((ao << 1) | (aol >> 31)) & bo) | (((bo << 1) | (bol >> 31)) & ao);
  }
  return st;
}

// Strip run holding tile pixel x of strip k (x must be set in the strip).
VL_DEV int sid(const CclSmem& s, int k, int x) {
  const int w = x >> 5;
  return s.base[k] + s.pre[k][w] + __popc(s.st[k][w] & le_mask(x & 31)) - 1;
}

VL_DEV bool mbit(const CclSmem& s, int row, int x) {
  return (s.m[row][x >> 5] >> (x & 31)) & 1u;
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

// Anchor of the boundary run starting at tile pixel x of boundary b: the
// strip run of its first pixel (upper strip if the upper row is set there).
VL_DEV int anchor_at(const CclSmem& s, int b, int x) {
  return mbit(s, 2 * b + 1, x) ? sid(s, b, x) : sid(s, b + 1, x);
}

// Root of strip run i once roots are encoded (parent[root] < 0).
VL_DEV int root_of(const CclSmem& s, int i) {
  const int p = s.parent[i];
  return p >= 0 ? p : i;
}

// Label one tile in shared memory.  Returns false (uniformly, after a block
// barrier) if the tile has more strip runs than the shared arrays hold, which
// cannot happen for CCL_TH x CCL_TWW tiles; the caller then skips the tile.
// On success: s.parent[i] of a non-root is its root (smallest id); a root
// holds a negative value, with `min_pixel` -(component's minimum linear pixel
// index + 2); s.flag[root] has bit0 when a seed pixel lies in the component
// (seed = mask and N phi1, if phi1 is given) and bit1 when the component
// reaches the tile border.  Must be called by every thread of the block.
// Rows of the tile into shared memory, strip unions, strip-run starts and
// their prefix counts.  Returns the number of strip runs (uniform, after a
// block barrier).
VL_DEV int ccl_tile_strips(CclSmem& s, const uint32_t* mask, const CclGeom& g, int conn) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = (g.th + 1) >> 1;
  // 1. rows, strip unions, strip-run starts, per-strip prefix counts
  for (int k = warp; k < ns; k += nw) {
    const int r0 = 2 * k, r1 = 2 * k + 1;
    uint32_t a = 0, b = 0;
    if (lane < g.tww) {
      // padding bits (columns >= W) are cleared here, so that no later pass
      // can see a pixel outside the image whatever the caller's buffer holds
      const uint32_t vm = vmask(g.w0 + lane, g.W);
      a = ldcg(&mask[(size_t)(g.r0 + r0) * g.Wp + g.w0 + lane]) & vm;
      if (r1 < g.th) b = ldcg(&mask[(size_t)(g.r0 + r1) * g.Wp + g.w0 + lane]) & vm;
    }
    uint32_t al = __shfl_up_sync(FULL, a, 1), bl = __shfl_up_sync(FULL, b, 1);
    if (lane == 0) al = bl = 0;
    const uint32_t st = strip_starts(a, b, al, bl, conn);
    const int c = __popc(st);
    const int incl = warp_incl_scan(c, lane);
    s.m[r0][lane] = a;
    s.m[r1][lane] = b;
    s.u[k][lane] = a | b;
    s.st[k][lane] = st;
    s.pre[k][lane] = incl - c;
    if (lane == 31) s.base[k + 1] = incl;
  }
  __syncthreads();
  if (warp == 0) {
    const int v = (lane < ns) ? s.base[lane + 1] : 0;
    const int incl = warp_incl_scan(v, lane);
    __syncwarp();
    if (lane < ns) s.base[lane] = incl - v;
    if (lane == 31) s.nruns = incl;
    if (lane == 31) s.base[ns] = incl;
  }
  __syncthreads();
  return s.nruns;
}

VL_DEV bool ccl_tile_label(CclSmem& s, const uint32_t* mask, const uint32_t* phi1,
                           const CclGeom& g, int conn, bool min_pixel, int32_t* status) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = (g.th + 1) >> 1;
  ccl_tile_strips(s, mask, g, conn);
  const int nruns = s.nruns;
  if (nruns > CCL_MAXRUNS) {  // uniform: every thread reads the same count
    set_status(status, ST_INTERNAL | RS_TRUNS);
    return false;
  }
  for (int i = tid; i < nruns; i += blockDim.x) {
    s.parent[i] = i;
    s.flag[i] = 0;
  }
  // 2. anchor of the boundary run entering each word from the left
  for (int b = warp; b < ns - 1; b += nw) {
    uint32_t A = 0, B = 0;
    if (lane < g.tww) { A = s.m[2 * b + 1][lane]; B = s.m[2 * b + 2][lane]; }
    uint32_t Al = __shfl_up_sync(FULL, A, 1), Bl = __shfl_up_sync(FULL, B, 1);
    if (lane == 0) Al = Bl = 0;
    const uint32_t qs = strip_starts(A, B, Al, Bl, conn);
    int last = -1;
    if (qs) last = anchor_at(s, b, 32 * lane + 31 - __clz(qs));
    int idx = last >= 0 ? lane : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, idx, o);
      if (lane >= o) idx = max(idx, t);
    }
    int prev = __shfl_up_sync(FULL, idx, 1);
    if (lane == 0) prev = -1;
    const int carried = __shfl_sync(FULL, last, prev < 0 ? 0 : prev);
    s.qc[b][lane] = prev < 0 ? -1 : carried;
  }
  __syncthreads();
  // 3. unite across strip boundaries, one tree level at a time (boundary b
  // belongs to level = trailing ones of b), so each level unites disjoint
  // groups of strips.  Every thread takes a share of the row-run starts
  // ("events") of one boundary word; the word's strip data sits in
  // registers.  In each round every thread with an event links its pair of
  // roots (atomicMin of the larger root's parent); a link that finds the
  // larger root already linked elsewhere leaves the follow-up union (old
  // parent, lo) to the same thread.
  const int cap = nruns + 64;
  bool ok = true;
  for (int level = 0; (1 << level) < ns; ++level) {
    const int step = 2 << level, first = (1 << level) - 1;  // b = first + j * step
    const int nb = (ns - 1 - first + step - 1) / step;
    const int pairs = nb > 0 ? nb * g.tww : 0;
    int T = 1;
    while (pairs > 0 && T * 2 * pairs <= (int)blockDim.x) T *= 2;
    const int pair = tid / T, sub = tid - (tid / T) * T;
    const bool act = pair < pairs;
    uint32_t A = 0, B = 0, qs = 0, evA = 0, evB = 0, stb = 0, stc = 0;
    int b = 0, w = 0, bb = 0, bc = 0, carry = -1;
    if (act) {
      b = first + (pair / g.tww) * step;
      w = pair - (pair / g.tww) * g.tww;
      A = s.m[2 * b + 1][w];
      B = s.m[2 * b + 2][w];
      const uint32_t Al = w > 0 ? s.m[2 * b + 1][w - 1] : 0u;
      const uint32_t Bl = w > 0 ? s.m[2 * b + 2][w - 1] : 0u;
      qs = strip_starts(A, B, Al, Bl, conn);
      stb = s.st[b][w];
      stc = s.st[b + 1][w];
      bb = s.base[b] + s.pre[b][w] - 1;
      bc = s.base[b + 1] + s.pre[b + 1][w] - 1;
      carry = s.qc[b][w];
      // one event per (boundary run, strip run): keep a row-run start only
      // when a boundary-run or strip-run start separates it from the
      // previous one, i.e. the first row-run start of every segment that
      // begins at such a start (or at the word's left edge)
      const uint32_t ra_ = A & ~((A << 1) | (Al >> 31));
      const uint32_t rb_ = B & ~((B << 1) | (Bl >> 31));
      evA = first_in_segments(ra_, qs | stb);
      evB = first_in_segments(rb_, qs | stc);
    }
    const int nA = __popc(evA), nE = nA + __popc(evB);
    // this thread's events: a contiguous share [j, e1) of the pair's list
    // (the A events, then the B events), walked by clearing lowest bits
    const int per = (nE + T - 1) / T;
    int j = min(nE, sub * per);
    const int e1 = min(nE, j + per);
    uint32_t curA = 0, curB = 0;
    if (j < e1) {
      if (j < nA) {
        curA = j ? evA & ~((1u << __fns(evA, 0, j + 1)) - 1u) : evA;
        curB = evB;
      } else {
        curB = j > nA ? evB & ~((1u << __fns(evB, 0, j - nA + 1)) - 1u) : evB;
      }
    }
    int pu = -1, pv = -1;
    for (int round = 0; round < 4 * CCL_MAXRUNS; ++round) {
      const bool has = act && (pu >= 0 || j < e1);
      if (!__any_sync(FULL, has)) break;
      int ra = 0, rb = 0;
      const bool from_event = has && pu < 0;
      if (has) {
        int u = pu, v = pv;
        if (from_event) {
          const bool isA = curA != 0;
          const uint32_t cur = isA ? curA : curB;
          const int p = __ffs(cur) - 1;
          if (isA) curA &= curA - 1u;
          else curB &= curB - 1u;
          u = isA ? bb + __popc(stb & le_mask(p)) : bc + __popc(stc & le_mask(p));
          const uint32_t qq = qs & le_mask(p);
          if (qq) {
            const int q = 31 - __clz(qq);
            v = ((A >> q) & 1u) ? bb + __popc(stb & le_mask(q)) : bc + __popc(stc & le_mask(q));
          } else {
            v = carry >= 0 ? carry : u;
          }
        }
        // both roots at once; walks that meet need no link
        ra = u; rb = v;
        if (!s_find2(s.parent, ra, rb, cap)) { ok = false; ra = rb = 0; }
      }
      // link the larger root under the smaller; when hi was no longer a
      // root its old parent (unless already lo) still has to meet lo
      const bool need = has && ra != rb;
      const int hi = max(ra, rb), lo = min(ra, rb);
      int old = hi;
      if (need) old = atomicMin(&s.parent[hi], lo);
      if (has) {
        if (from_event) ++j;
        else pu = pv = -1;
        if (need && old != hi && old != lo) { pu = old; pv = lo; }
      }
    }
    __syncthreads();
    // (no flatten between levels: path halving in s_find keeps the next
    // level's walks short, and a full pass over all runs costs more)
  }
  // 4. flatten: every thread points its own runs at their roots with finds
  // that only read.  (A path-halving find writes grandparents into the
  // entries it passes; landing after another thread's final write to one of
  // them, such a write would leave that run one hop short of its root.)
  // Other threads' writes only move entries closer to the roots, so a
  // read-only walk still ends at the root.
  {
    volatile int32_t* vp = s.parent;
    for (int i = tid; i < nruns; i += blockDim.x) {
      int x = i, it = 0;
      for (; it < cap; ++it) {
        const int q = vp[x];
        if (q == x) break;
        if ((unsigned)q >= (unsigned)nruns) { it = cap; break; }
        x = q;
      }
      if (it == cap) { ok = false; x = i; }
      vp[i] = x;
    }
  }
  if (!ok) set_status(status, ST_INTERNAL | RS_SUNION);
  __syncthreads();
  // roots now hold their (to be minimised) representative, encoded negative
  for (int i = tid; i < nruns; i += blockDim.x)
    if (s.parent[i] == i) s.parent[i] = INT_MIN;
  __syncthreads();
  // 5. seeds: components holding a pixel of mask and N phi1
  if (phi1 != nullptr) {
    for (int r = warp; r < g.th; r += nw) {
      uint32_t z = warp_near_row(phi1, g.H, g.W, g.Wp, g.r0 + r, g.w0, lane, g.tww, conn);
      z &= s.m[r][lane];
      uint32_t zl = __shfl_up_sync(FULL, z, 1);
      if (lane == 0) zl = 0;
      uint32_t zs = z & ~((z << 1) | (zl >> 31));
      while (zs) {
        const int p = __ffs(zs) - 1;
        zs &= zs - 1;
        s.flag[root_of(s, sid(s, r >> 1, 32 * lane + p))] = 1;
      }
    }
    __syncthreads();
  }
  // 6. components on the tile border (rows 0 and th-1, first/last column)
  for (int k = warp; k < ns; k += nw) {
    if (lane < g.tww) {
      for (int r = 2 * k; r <= 2 * k + 1; ++r) {
        if (r != 0 && r != g.th - 1) continue;
        const uint32_t m = s.m[r][lane];
        uint32_t rs = m & ~((m << 1) | (lane > 0 ? (s.m[r][lane - 1] >> 31) : 0u));
        while (rs) {
          const int p = __ffs(rs) - 1;
          rs &= rs - 1;
          s.flag[root_of(s, sid(s, k, 32 * lane + p))] |= 2;
        }
      }
      const uint32_t u = s.u[k][lane];
      if (lane == 0 && (u & 1u)) s.flag[root_of(s, s.base[k])] |= 2;
      if (lane == g.tww - 1 && (u >> 31)) s.flag[root_of(s, s.base[k + 1] - 1)] |= 2;
    }
  }
  // 7. minimum pixel of each component (for canonical labels): only strip
  // runs in the component's first strip can hold it
  if (min_pixel) {
    for (int k = warp; k < ns; k += nw) {
      if (lane >= g.tww) continue;
      uint32_t sc = s.st[k][lane];
      while (sc) {
        const int p = __ffs(sc) - 1;
        sc &= sc - 1;
        const int x = 32 * lane + p;
        const int S = sid(s, k, x);
        const int R = root_of(s, S);
        if (R < s.base[k]) continue;
        // first pixel of the top row inside this strip run, else its start
        int best = -1;
        for (int ww = lane, pp = p; ww < g.tww; ++ww, pp = 0) {
          const uint32_t from = ~(le_mask(pp) >> 1);  // bits >= pp
          const uint32_t u = s.u[k][ww];
          // the run ends at the first zero of u or the next run start
          uint32_t stop = (~u | (s.st[k][ww] & ~(ww == lane ? le_mask(p) : 0u))) & from;
          if (ww == lane) stop &= ~(1u << p);
          const uint32_t ext = stop ? (from & ((stop & (0u - stop)) - 1u)) : from;
          const uint32_t hit = s.m[2 * k][ww] & ext;
          if (hit) { best = 32 * ww + __ffs(hit) - 1; break; }
          if (stop) break;
        }
        const int row = best >= 0 ? 2 * k : 2 * k + 1;
        const int col = best >= 0 ? best : x;
        atomicMax(&s.parent[R], -((g.r0 + row) * g.W + 32 * g.w0 + col + 2));
      }
    }
  }
  __syncthreads();
  return true;
}

// Per-tile storage between the local and the final pass: the encoded
// union-find state (non-roots: their root; roots: -(representative + 2))
// and the component flags.  The final pass rebuilds the strips from the mask
// and reloads this instead of labelling the tile again.
VL_DEV int ccl_tile_cap(int Wp, int cth = CCL_TH) { return (cth / 2) * min(CCL_TWW, Wp) * 32; }

VL_DEV void ccl_tile_save(const CclSmem& s, int32_t* tpar, uint8_t* tflag) {
  for (int i = threadIdx.x; i < s.nruns; i += blockDim.x) {
    tpar[i] = s.parent[i];
    tflag[i] = s.flag[i];
  }
}

VL_DEV bool ccl_tile_load(CclSmem& s, const uint32_t* mask, const CclGeom& g, int conn,
                          const int32_t* tpar, const uint8_t* tflag, int32_t* status) {
  const int n = ccl_tile_strips(s, mask, g, conn);
  if (n > CCL_MAXRUNS) {
    set_status(status, ST_INTERNAL | RS_TRUNS);
    return false;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int v = ldcg(tpar + i);
    if (v >= n) {  // never written by a successful local pass: keep indexes in range
      set_status(status, ST_INTERNAL | RS_TLOAD);
      v = -2;
    }
    s.parent[i] = v;
    s.flag[i] = ldcg(tflag + i);
  }
  __syncthreads();
  return true;
}

// Encoded value of the root of strip run i (see ccl_encode_roots).
VL_DEV int root_value(const CclSmem& s, int i) {
  int p = s.parent[i];
  if (p >= 0) p = s.parent[p];
  return -p - 2;
}
// Value at tile pixel (row r, column x), which must be set.
VL_DEV int pixel_value(const CclSmem& s, int r, int x) {
  return root_value(s, sid(s, r >> 1, x));
}

// Modes of ccl_encode_roots.
constexpr int ENC_PUBLISH = 0;     // labels: value = minimum pixel; publish border roots
constexpr int ENC_PUBLISH_RZ = 1;  // rho: value = key (below); publish border roots
constexpr int ENC_LABEL = 2;       // value = global label (border roots resolved in G)
constexpr int ENC_SELECT = 3;      // flag bit2 = component selected (rho)

// Keys of the component select.  A tile-local component is keyed by the
// first pixel v of its root strip run when it holds a seed pixel, and by
// v + npx when it does not; G then has 2 * npx entries.  The global merge
// links the larger root under the smaller, so a merged component's root is
// a seeded key (< npx) exactly when one of its parts was seeded: the seed
// flag travels with the union itself and no separate pass has to gather it.
VL_DEV int rz_key(int v, bool seeded, int npx) { return seeded ? v : v + npx; }

// Give every local root its value.  The publishing modes visit each root
// once, at its start pixel, and replace parent[root] by -(value + 2); the
// resolving modes (ENC_LABEL, ENC_SELECT) start from the saved values and
// walk G for the roots of border components only.  Block barrier at the end.
//   ENC_PUBLISH     value = the component's minimum pixel (computed by the
//                   labelling); border components publish G[value] = value
//   ENC_PUBLISH_RZ  value = rz_key of the first pixel of the root strip run;
//                   border components publish G[value] = value
//   ENC_LABEL       value = the global root of the saved value (border
//                   components), else the saved value
//   ENC_SELECT      flag bit2 set when the component is selected: seeded
//                   locally, or its global root is a seeded key
// glen: entries of G (npx for labels, 2 * npx for rho).  Finds compress
// their paths: a node only ever moves to an ancestor, and in the labelling
// the final label of every node on a path is the root it is moved to.
VL_DEV void ccl_encode_roots(CclSmem& s, const CclGeom& g, int mode, int32_t* G, int glen,
                             int npx, int32_t* status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = (g.th + 1) >> 1;
  if (mode == ENC_LABEL || mode == ENC_SELECT) {
    // the saved roots already hold their value: only the components on the
    // tile border have work, a walk in G.  The strip runs are dealt out over
    // every thread of the block, so the walks of one tile run side by side
    // (the border components' roots sit in the first and last strips).
    for (int i = threadIdx.x; i < s.nruns; i += blockDim.x) {
      const int p = s.parent[i];
      if (p >= 0) continue;  // not a root
      const uint8_t fl = s.flag[i];
      if (mode == ENC_LABEL) {
        if (fl & 2) s.parent[i] = -(g_find(G, -p - 2, glen, status) + 2);
      } else {
        const bool sel = (fl & 2) ? g_find(G, -p - 2, glen, status) < npx : (fl & 1) != 0;
        if (sel) s.flag[i] = fl | 4;
      }
    }
    __syncthreads();
    return;
  }
  for (int k = warp; k < ns; k += nw) {
    if (lane >= g.tww) continue;
    uint32_t sc = s.st[k][lane];
    while (sc) {
      const int p = __ffs(sc) - 1;
      sc &= sc - 1;
      const int x = 32 * lane + p;
      const int S = sid(s, k, x);
      if (s.parent[S] >= 0) continue;  // not a root
      const uint8_t fl = s.flag[S];
      int v;
      if (mode == ENC_PUBLISH_RZ) {
        v = rz_key((g.r0 + (mbit(s, 2 * k, x) ? 2 * k : 2 * k + 1)) * g.W + 32 * g.w0 + x,
                   fl & 1, npx);
      } else {
        v = -s.parent[S] - 2;
      }
      if (fl & 2) G[v] = v;
      s.parent[S] = -(v + 2);
    }
  }
  __syncthreads();
}

// Border pixels of the tile point at their component's representative in G.
VL_DEV void ccl_publish_border(CclSmem& s, const CclGeom& g, int32_t* G) {
  const int width = 32 * g.tww;
  const int n = 2 * width + 2 * g.th;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int r, x;
    if (i < width) { r = 0; x = i; }
    else if (i < 2 * width) { r = g.th - 1; x = i - width; }
    else if (i < 2 * width + g.th) { r = i - 2 * width; x = 0; }
    else { r = i - 2 * width - g.th; x = width - 1; }
    if (mbit(s, r, x)) G[(g.r0 + r) * g.W + 32 * g.w0 + x] = pixel_value(s, r, x);
  }
}

// Write labels of the tile (after ENC_LABEL).  First every strip run takes
// its root's encoded value (after the flatten non-roots point at roots, and
// roots are not written, so the pass needs no ordering), then each lane
// writes 4 consecutive pixels per step: a warp covers 128 pixels of a row
// with 16-byte stores when rows are 16-byte aligned.
VL_DEV void ccl_write_labels(CclSmem& s, const CclGeom& g, int32_t* labels) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < s.nruns; i += blockDim.x) {
    const int p = s.parent[i];
    if (p >= 0) s.parent[i] = s.parent[p];
  }
  __syncthreads();
  const int x_end = min(32 * g.tww, g.W - 32 * g.w0);
  const bool vec = (g.W & 3) == 0;
  for (int r = warp; r < g.th; r += nw) {
    int32_t* row = labels + (size_t)(g.r0 + r) * g.W + 32 * g.w0;
    const int k = r >> 1;
    for (int x0 = 4 * lane; x0 < x_end; x0 += 128) {
      const int w = x0 >> 5, b = x0 & 31;
      const uint32_t bits = s.m[r][w] >> b;
      const uint32_t st = s.st[k][w];
      const int base = s.base[k] + s.pre[k][w] - 1;
      int v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        v[q] = ((bits >> q) & 1u) ? -s.parent[base + __popc(st & le_mask(b + q))] - 2 : -1;
      if (vec && x0 + 4 <= x_end) {
        *reinterpret_cast<int4*>(row + x0) = make_int4(v[0], v[1], v[2], v[3]);
      } else {
        for (int q = 0; q < 4 && x0 + q < x_end; ++q) row[x0 + q] = v[q];
      }
    }
  }
}

// Write Z = the selected components of the tile (after ENC_SELECT).
VL_DEV void ccl_write_select(const CclSmem& s, const CclGeom& g, uint32_t* Z) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = (g.th + 1) >> 1;
  for (int k = warp; k < ns; k += nw) {
    if (lane >= g.tww) continue;
    const uint32_t u = s.u[k][lane], st = s.st[k][lane];
    uint32_t f = 0, sc = st;
    while (sc) {
      const int p = __ffs(sc) - 1;
      sc &= sc - 1;
      if (s.flag[root_of(s, sid(s, k, 32 * lane + p))] & 4) f |= 1u << p;
    }
    // a run entering from the left word continues through bit 0
    const uint32_t e = u & ~st;
    const uint32_t inj = (f << 1) | ((e & 1u) && (s.flag[root_of(s, sid(s, k, 32 * lane))] & 4) ? 1u : 0u);
    // carry through the continuation bits of each selected run
    const uint32_t sel = f | (((e + inj) ^ e) & e);
    for (int r = 2 * k; r <= 2 * k + 1 && r < g.th; ++r)
      Z[(size_t)(g.r0 + r) * g.Wp + g.w0 + lane] = s.m[r][lane] & sel;
  }
}

// --------------------------------------------------------- border merge --
// The borders between labelling tiles are merged by a pass of their own
// after the labelling launch, in merge units: one per word of each
// horizontal tile border (its 32 columns) and one per 32 rows of each
// vertical tile border.  A warp takes a unit, one lane per column (or row),
// so the unions of a unit run side by side.  (A merge inside the labelling
// launch, by whichever tile beside a border finished last, measured slower:
// its latency-bound walks then hold a labelling CTA instead of running at
// full occupancy.)

// Which of columns x-1, x, x+1 (8-adjacency) or x (4-adjacency) of a row is
// set, leftmost first, as an offset -1/0/1 (2: none).  The row is given by
// the words left of, at, and right of x's word (0 outside the image), and
// b = x mod 32.
VL_DEV int window_hit(uint32_t l, uint32_t c, uint32_t r, int b, int conn) {
  if (conn == 8) {
    const uint32_t left = b > 0 ? (c >> (b - 1)) & 1u : (l >> 31);
    if (left) return -1;
    if ((c >> b) & 1u) return 0;
    const uint32_t right = b < 31 ? (c >> (b + 1)) & 1u : (r & 1u);
    return right ? 1 : 2;
  }
  return ((c >> b) & 1u) ? 0 : 2;
}

// Every lane offers at most one pixel pair (a, b) across a tile border.  The
// pairs become pairs of component keys (border pixels hold their component's
// representative in G, so a plain read gives a key without a find); equal
// key pairs in the warp are united once, by the lowest lane holding them.
// Must be called by the whole warp.
VL_DEV void warp_unite(int32_t* G, bool valid, int a, int b, int glen, int32_t* status) {
  int ka = 0, kb = 0;
  if (valid) {
    ka = ldcg(&G[a]);
    kb = ldcg(&G[b]);
    valid = ka != kb;
  }
  const unsigned long long key =
      valid ? (((unsigned long long)(unsigned)max(ka, kb) << 32) | (unsigned)min(ka, kb)) : ~0ull;
  const unsigned peers = __match_any_sync(FULL, key);
  if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) g_union(G, ka, kb, glen, status);
}

// Two pairs per lane, (a1, b1) and (a2, b2).  When the warp holds at most 32
// valid pairs they are dealt out one per lane, so the unions run side by
// side in one round instead of two.  Must be called by the whole warp.
VL_DEV void warp_unite2(int32_t* G, bool v1, int a1, int b1, bool v2, int a2, int b2, int glen,
                        int32_t* status) {
  const int lane = threadIdx.x & 31;
  const unsigned m1 = __ballot_sync(FULL, v1), m2 = __ballot_sync(FULL, v2);
  const int n1 = __popc(m1), n = n1 + __popc(m2);
  if (n > 32) {
    warp_unite(G, v1, a1, b1, glen, status);
    warp_unite(G, v2, a2, b2, glen, status);
    return;
  }
  // lane L takes the L-th valid pair: the first kind's in lane order, then
  // the second's
  int src = lane;
  if (lane < n1) src = __fns(m1, 0, lane + 1);
  else if (lane < n) src = __fns(m2, 0, lane - n1 + 1);
  const int xa1 = __shfl_sync(FULL, a1, src), xb1 = __shfl_sync(FULL, b1, src);
  const int xa2 = __shfl_sync(FULL, a2, src), xb2 = __shfl_sync(FULL, b2, src);
  const bool first = lane < n1;
  warp_unite(G, lane < n, first ? xa1 : xa2, first ? xb1 : xb2, glen, status);
}

// Unite the components of row yu and row yd (rows of the stored image) that
// touch in word w: with conn 8 a pixel meets the three pixels at x - 1, x,
// x + 1 of the other row, with conn 4 only the one at x.  Every row-run
// start of either row is checked against that window of the other row: two
// runs that touch always have a start of one run inside the other's window.
// Padding bits are cleared.  Must be called by the whole warp.
VL_DEV void ccl_merge_rows(const uint32_t* m, int W, int Wp, int yu, int yd, int w, int conn,
                           int32_t* G, int glen, int32_t* status) {
  const int lane = threadIdx.x & 31;
  uint32_t v = 0;
  if (lane < 6) {
    const int ww = w - 1 + lane % 3;
    if (ww >= 0 && ww < Wp) v = ldcg(&m[(size_t)(lane < 3 ? yu : yd) * Wp + ww]) & vmask(ww, W);
  }
  const uint32_t mul = __shfl_sync(FULL, v, 0), mu = __shfl_sync(FULL, v, 1),
                 mur = __shfl_sync(FULL, v, 2), mdl = __shfl_sync(FULL, v, 3),
                 md = __shfl_sync(FULL, v, 4), mdr = __shfl_sync(FULL, v, 5);
  const uint32_t sd = md & ~((md << 1) | (mdl >> 31));
  const uint32_t su = mu & ~((mu << 1) | (mul >> 31));
  const int x = 32 * w + lane;
  const int dd = (sd >> lane) & 1u ? window_hit(mul, mu, mur, lane, conn) : 2;
  const int du = (su >> lane) & 1u ? window_hit(mdl, md, mdr, lane, conn) : 2;
  warp_unite2(G, dd != 2, yd * W + x, yu * W + x + dd, du != 2, yu * W + x, yd * W + x + du,
              glen, status);
}

// (Hs: slice rows of a volume, H for an image; horizontal borders are those
// between the tile rows of one slice.)
VL_DEV int merge_units(int H, int Wp, int tiles_x, int Hs, int cth = CCL_TH) {
  const int tys = (Hs + cth - 1) / cth;
  return (H / Hs) * (tys - 1) * Wp + (tiles_x - 1) * ((H + 31) >> 5);
}

// Unite the components that touch across the tile border of merge unit
// `unit`.  A horizontal border is ccl_merge_rows over the whole row.  A
// vertical border pairs each set pixel left of it with the pixel right of it,
// or, for 8-adjacency when that one is clear, with its diagonal neighbours
// (both border columns lie inside the image: a tile border is a multiple of
// 1024 columns, below W).  Must be called by the whole warp.
VL_DEV void ccl_merge_unit(const uint32_t* m, int H, int W, int Wp, int unit, int conn,
                           int32_t* G, int glen, int32_t* status, int Hs, int cth = CCL_TH) {
  const int lane = threadIdx.x & 31;
  const int tys = (Hs + cth - 1) / cth;
  const int nh = (H / Hs) * (tys - 1) * Wp;
  if (unit < nh) {
    const int border = unit / Wp, w = unit - border * Wp;  // border: over all slices
    const int z = border / (tys - 1), k = border - z * (tys - 1) + 1;
    const int yd = z * Hs + k * cth, yu = yd - 1;
    ccl_merge_rows(m, W, Wp, yu, yd, w, conn, G, glen, status);
  } else {
    const int nv = (H + 31) >> 5;
    const int j = unit - nh;
    const int kk = j / nv + 1;
    const int y = (j - (kk - 1) * nv) * 32 + lane;
    const int x0 = kk * CCL_TWW * 32;  // first column right of the border (< W)
    const int wl = (x0 - 1) >> 5, wr = x0 >> 5;
    uint32_t L = 0, R = 0, Ru = 0, Rd = 0;
    if (y < H) {
      L = ldcg(&m[(size_t)y * Wp + wl]) >> 31;
      R = ldcg(&m[(size_t)y * Wp + wr]) & 1u;
    }
    if (conn == 8) {
      Ru = __shfl_up_sync(FULL, R, 1);
      Rd = __shfl_down_sync(FULL, R, 1);
      if (lane == 0) Ru = (y > 0 && y - 1 < H) ? ldcg(&m[(size_t)(y - 1) * Wp + wr]) & 1u : 0u;
      if (lane == 31) Rd = (y + 1 < H) ? ldcg(&m[(size_t)(y + 1) * Wp + wr]) & 1u : 0u;
      // diagonals stay inside one slice of a volume
      if (y % Hs == 0) Ru = 0;
      if ((y + 1) % Hs == 0) Rd = 0;
    }
    // (lane-dependent choices go into the arguments: every lane calls)
    const int a = y * W + x0 - 1;
    const bool straight = R || conn == 4;
    warp_unite2(G, L && (straight ? R : Ru), a, (straight ? y : y - 1) * W + x0,
                L && !straight && Rd, a, (y + 1) * W + x0, glen, status);
  }
}

}  // namespace vl
