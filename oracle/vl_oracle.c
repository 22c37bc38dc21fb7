/*
 * Reference evaluator for SLCS formulas on 2D images -- TEST INFRASTRUCTURE.
 *
 * This file is the oracle that the CUDA library is checked against.  It is
 * deliberately plain and slow: one byte per pixel, literal loops, BFS.  It
 * shares no code, header or constant with the CUDA path; only tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Semantics followed (paper: "A spatial model checker in GPU", Sec. 2):
 *   - the model is a 2D image of fixed size; a formula denotes the set of
 *     pixels satisfying it, i.e. a binary image (Sec. 2);
 *   - atomic propositions are thresholds on an image feature (Sec. 2; the
 *     spec of Fig. "specification" uses intensity(img) >. c), compared in
 *     float32, strictly;
 *   - not / and are pixel-wise complement / intersection (Sec. 2);
 *   - N phi is the set of pixels sharing a vertex or an edge with a phi pixel
 *     (Moore neighbourhood), i.e. the dilation of phi (Sec. 2); read as
 *     reflexive, clipped at the image border; with 4-adjacency the cross is
 *     used instead;
 *   - rho phi1[phi2] is the set of x with a path pi, an index l, pi_0 = x,
 *     pi_l |= phi1 and pi_1..pi_{l-1} |= phi2 (Sec. 2); computed by a BFS
 *     backwards from phi1 through phi2 pixels;
 *   - connected components: flood fill, each component labelled by its
 *     minimum linear index y*W + x, background -1;
 *   - percentile of a channel: the value at rank floor(q (n-1)) of the
 *     ascending sort of its n = H*W values (the "percentiles" normalisation
 *     of Sec. 4.2; no interpolation); NaN values sort after +infinity;
 *   - number terms (basic arithmetic beside the SLCS primitives, Sec. 3):
 *     VALUE reads an image channel as numbers; ADD, SUB, MUL, DIV combine
 *     two terms (or a term and a float32 constant) pixel by pixel in
 *     IEEE-754 binary32, round to nearest even, each result stored as a
 *     float before the next operation uses it.  Thresholds and percentiles
 *     may compare a number term instead of an image channel.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define VLO_EXPORT __attribute__((visibility("default")))

/* ---------------------------------------------------------------- atoms -- */

VLO_EXPORT void vlo_threshold(const float* img, int64_t n, float t, int gt,
                              uint8_t* out) {
  for (int64_t i = 0; i < n; ++i) {
    float v = img[i];
    out[i] = gt ? (v > t) : (v < t);
  }
}

/* -------------------------------------------------------------- boolean -- */

VLO_EXPORT void vlo_not(const uint8_t* a, int64_t n, uint8_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = a[i] ? 0 : 1;
}

VLO_EXPORT void vlo_and(const uint8_t* a, const uint8_t* b, int64_t n,
                        uint8_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (a[i] && b[i]) ? 1 : 0;
}

/* ------------------------------------------------------------ neighbours -- */

/* Is (y+dy, x+dx) a neighbour of (y, x) under the given adjacency?  The pixel
 * itself counts (N is read as reflexive). */
static int is_offset(int dy, int dx, int conn) {
  if (dy < -1 || dy > 1 || dx < -1 || dx > 1) return 0;
  if (conn == 4) return (dy == 0) || (dx == 0);
  return 1;
}

/* N phi: OR of phi over the (clipped) neighbourhood of each pixel. */
VLO_EXPORT void vlo_near(const uint8_t* a, int H, int W, int conn,
                         uint8_t* out) {
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      uint8_t v = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!is_offset(dy, dx, conn)) continue;
          int yy = y + dy, xx = x + dx;
          if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
          if (a[(int64_t)yy * W + xx]) v = 1;
        }
      out[(int64_t)y * W + x] = v;
    }
}

/* ---------------------------------------------------------- reachability -- */

/* rho phi1[phi2].  R starts as phi1 (the l = 0 case).  A pixel is "expanded"
 * when it is in phi1, or it is a phi2 pixel in R.  Every neighbour of an
 * expanded pixel is in R: it is pi_0 of a path whose pi_1 is the expanded
 * pixel.  Returns 0, or -1 when memory runs out. */
VLO_EXPORT int vlo_reach(const uint8_t* phi1, const uint8_t* phi2, int H,
                         int W, int conn, uint8_t* out) {
  int64_t n = (int64_t)H * W;
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  uint8_t* pushed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!queue || !pushed) { free(queue); free(pushed); return -1; }
  int64_t head = 0, tail = 0;
  for (int64_t i = 0; i < n; ++i) {
    out[i] = phi1[i] ? 1 : 0;
    if (phi1[i]) { queue[tail++] = i; pushed[i] = 1; }
  }
  while (head < tail) {
    int64_t v = queue[head++];
    int y = (int)(v / W), x = (int)(v % W);
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dy == 0 && dx == 0) continue;
        if (!is_offset(dy, dx, conn)) continue;
        int yy = y + dy, xx = x + dx;
        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
        int64_t u = (int64_t)yy * W + xx;
        out[u] = 1;                       /* u = pi_0, v = pi_1 */
        if (phi2[u] && !pushed[u]) {      /* u may serve as an intermediate */
          pushed[u] = 1;
          queue[tail++] = u;
        }
      }
  }
  free(queue);
  free(pushed);
  return 0;
}

/* ---------------------------------------------------------- components -- */

/* Flood fill in raster order.  The first pixel met of each component is its
 * minimum linear index, which becomes its label.  Background gets -1.
 * Returns the number of components, or -1 when memory runs out. */
VLO_EXPORT int64_t vlo_ccl(const uint8_t* m, int H, int W, int conn,
                           int32_t* labels) {
  int64_t n = (int64_t)H * W;
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!queue) return -1;
  for (int64_t i = 0; i < n; ++i) labels[i] = -1;
  int64_t count = 0;
  for (int64_t s = 0; s < n; ++s) {
    if (!m[s] || labels[s] != -1) continue;
    ++count;
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    labels[s] = (int32_t)s;
    while (head < tail) {
      int64_t v = queue[head++];
      int y = (int)(v / W), x = (int)(v % W);
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dy == 0 && dx == 0) continue;
          if (!is_offset(dy, dx, conn)) continue;
          int yy = y + dy, xx = x + dx;
          if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
          int64_t u = (int64_t)yy * W + xx;
          if (m[u] && labels[u] == -1) {
            labels[u] = (int32_t)s;
            queue[tail++] = u;
          }
        }
    }
  }
  free(queue);
  return count;
}

/* ----------------------------------------------------------- percentile -- */

/* Ascending order with every NaN after +infinity (NaNs equal). */
static int cmp_float(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  int nx = x != x, ny = y != y;
  if (nx || ny) return nx - ny;
  return (x > y) - (x < y);
}

/* Value at rank floor(q * (n - 1)) of the ascending sort (q clamped to
 * [0, 1]).  Returns 0 for n == 0. */
VLO_EXPORT float vlo_percentile(const float* img, int64_t n, double q) {
  if (n <= 0) return 0.0f;
  float* v = (float*)malloc(sizeof(float) * (size_t)n);
  if (!v) return 0.0f;
  memcpy(v, img, sizeof(float) * (size_t)n);
  qsort(v, (size_t)n, sizeof(float), cmp_float);
  if (q < 0.0) q = 0.0;
  if (q > 1.0) q = 1.0;
  int64_t k = (int64_t)(q * (double)(n - 1)); /* floor for q >= 0 */
  if (k < 0) k = 0;
  if (k > n - 1) k = n - 1;
  float r = v[k];
  free(v);
  return r;
}

/* ------------------------------------------------------------ arithmetic -- */

enum { VLO_ARITH_ADD = 0, VLO_ARITH_SUB = 1, VLO_ARITH_MUL = 2, VLO_ARITH_DIV = 3 };

/* out[i] = a[i] (op) b[i], or a[i] (op) c when b is NULL; every result is
 * rounded to float by the store. */
VLO_EXPORT void vlo_arith(int op, const float* a, const float* b, float c, int64_t n,
                          float* out) {
  for (int64_t i = 0; i < n; ++i) {
    float x = a[i], y = b ? b[i] : c, r;
    switch (op) {
      case VLO_ARITH_ADD: r = x + y; break;
      case VLO_ARITH_SUB: r = x - y; break;
      case VLO_ARITH_MUL: r = x * y; break;
      default: r = x / y; break;
    }
    out[i] = r;
  }
}

/* ------------------------------------------------------- DAG evaluation -- */

/* Primitive operators only: derived connectives are expanded before a DAG
 * reaches this evaluator. */
enum {
  VLO_TRUE = 0, VLO_FALSE = 1, VLO_THR_GT = 2, VLO_THR_LT = 3,
  VLO_PCT_GT = 4, VLO_PCT_LT = 5, VLO_MASK = 6, VLO_NOT = 7, VLO_AND = 8,
  VLO_NEAR = 9, VLO_REACH = 10, VLO_VALUE = 16, VLO_ADD = 17, VLO_SUB = 18,
  VLO_MUL = 19, VLO_DIV = 20
};

typedef struct {
  int32_t op, a, b, image, channel;
  float t;
  double q;
} vlo_node;

static int is_number_op(int op) {
  return op == VLO_VALUE || op == VLO_ADD || op == VLO_SUB || op == VLO_MUL || op == VLO_DIV;
}

/* Number of operands (node indexes) of a node.  Thresholds and percentiles
 * have one when they compare a number term (a >= 0); an arithmetic node with
 * b < 0 takes the constant t as its second operand. */
static int node_arity(const vlo_node* d) {
  switch (d->op) {
    case VLO_NOT: case VLO_NEAR: return 1;
    case VLO_AND: case VLO_REACH: return 2;
    case VLO_THR_GT: case VLO_THR_LT: case VLO_PCT_GT: case VLO_PCT_LT: return d->a >= 0 ? 1 : 0;
    case VLO_ADD: case VLO_SUB: case VLO_MUL: case VLO_DIV: return d->b >= 0 ? 2 : 1;
    default: return 0;
  }
}

/* Evaluate a primitive DAG in index order.  images[i] is a float32 planar
 * (C, H, W) array; masks[i] a uint8 (H, W) array (for MASK atoms, indexed by
 * node.image).  out_roots[r] receives the (H, W) uint8 mask of roots[r].
 * Number terms are float (H, W) arrays.  Intermediate values are freed
 * after their last consumer.  Returns 0, -1 on malformed input, -2 when
 * memory runs out. */
VLO_EXPORT int vlo_eval(const vlo_node* nodes, int n_nodes, const int32_t* roots,
                        int n_roots, const float* const* images, int n_images,
                        int C, const uint8_t* const* masks, int n_masks, int H,
                        int W, int conn, uint8_t* const* out_roots) {
  int64_t n = (int64_t)H * W;
  if (n_nodes < 0 || n_roots < 0 || (conn != 4 && conn != 8)) return -1;
  void** val = (void**)calloc((size_t)(n_nodes > 0 ? n_nodes : 1), sizeof(void*));
  int32_t* uses = (int32_t*)calloc((size_t)(n_nodes > 0 ? n_nodes : 1), sizeof(int32_t));
  if (!val || !uses) { free(val); free(uses); return -2; }
  int rc = 0;
  for (int i = 0; i < n_nodes; ++i) {
    const vlo_node* d = &nodes[i];
    int arity = node_arity(d);
    if (arity >= 1 && (d->a < 0 || d->a >= i)) { rc = -1; goto done; }
    if (arity == 2 && (d->b < 0 || d->b >= i)) { rc = -1; goto done; }
    /* operand kinds: arithmetic and compared terms are numbers, the rest masks */
    int want_num = is_number_op(d->op) || d->op == VLO_THR_GT || d->op == VLO_THR_LT ||
                   d->op == VLO_PCT_GT || d->op == VLO_PCT_LT;
    if (arity >= 1 && is_number_op(nodes[d->a].op) != want_num) { rc = -1; goto done; }
    if (arity == 2 && is_number_op(nodes[d->b].op) != want_num) { rc = -1; goto done; }
    if (arity >= 1) uses[d->a]++;
    if (arity == 2) uses[d->b]++;
  }
  for (int r = 0; r < n_roots; ++r) {
    if (roots[r] < 0 || roots[r] >= n_nodes || is_number_op(nodes[roots[r]].op)) { rc = -1; goto done; }
  }
  for (int i = 0; i < n_nodes; ++i) {
    const vlo_node* d = &nodes[i];
    size_t bytes = (size_t)(n > 0 ? n : 1) * (is_number_op(d->op) ? sizeof(float) : 1);
    void* ov = malloc(bytes);
    if (!ov) { rc = -2; goto done; }
    val[i] = ov;
    uint8_t* o = (uint8_t*)ov;
    float* fo = (float*)ov;
    switch (d->op) {
      case VLO_TRUE: memset(o, 1, (size_t)n); break;
      case VLO_FALSE: memset(o, 0, (size_t)n); break;
      case VLO_THR_GT:
      case VLO_THR_LT:
      case VLO_PCT_GT:
      case VLO_PCT_LT: {
        const float* ch;
        if (d->a >= 0) {
          ch = (const float*)val[d->a];
        } else {
          if (d->image < 0 || d->image >= n_images || d->channel < 0 ||
              d->channel >= C) { rc = -1; goto done; }
          ch = images[d->image] + (int64_t)d->channel * n;
        }
        float t = d->t;
        if (d->op == VLO_PCT_GT || d->op == VLO_PCT_LT)
          t = vlo_percentile(ch, n, d->q);
        int gt = (d->op == VLO_THR_GT || d->op == VLO_PCT_GT);
        vlo_threshold(ch, n, t, gt, o);
        break;
      }
      case VLO_VALUE:
        if (d->image < 0 || d->image >= n_images || d->channel < 0 ||
            d->channel >= C) { rc = -1; goto done; }
        memcpy(fo, images[d->image] + (int64_t)d->channel * n, sizeof(float) * (size_t)n);
        break;
      case VLO_ADD: case VLO_SUB: case VLO_MUL: case VLO_DIV:
        vlo_arith(d->op - VLO_ADD, (const float*)val[d->a],
                  d->b >= 0 ? (const float*)val[d->b] : NULL, d->t, n, fo);
        break;
      case VLO_MASK:
        if (d->image < 0 || d->image >= n_masks) { rc = -1; goto done; }
        for (int64_t k = 0; k < n; ++k) o[k] = masks[d->image][k] ? 1 : 0;
        break;
      case VLO_NOT: vlo_not((const uint8_t*)val[d->a], n, o); break;
      case VLO_AND: vlo_and((const uint8_t*)val[d->a], (const uint8_t*)val[d->b], n, o); break;
      case VLO_NEAR: vlo_near((const uint8_t*)val[d->a], H, W, conn, o); break;
      case VLO_REACH:
        if (vlo_reach((const uint8_t*)val[d->a], (const uint8_t*)val[d->b], H, W, conn, o) != 0) {
          rc = -2;
          goto done;
        }
        break;
      default: rc = -1; goto done;
    }
    for (int r = 0; r < n_roots; ++r)
      if (roots[r] == i) memcpy(out_roots[r], o, (size_t)n);
    /* release operands whose last consumer was this node */
    int arity = node_arity(d);
    if (arity >= 1) uses[d->a]--;
    if (arity == 2) uses[d->b]--;
    if (arity >= 1 && uses[d->a] == 0 && val[d->a]) { free(val[d->a]); val[d->a] = NULL; }
    if (arity == 2 && uses[d->b] == 0 && val[d->b]) { free(val[d->b]); val[d->b] = NULL; }
    if (uses[i] == 0) { free(val[i]); val[i] = NULL; }
  }
done:
  for (int i = 0; i < n_nodes; ++i) free(val[i]);
  free(val);
  free(uses);
  return rc;
}

/* ------------------------------------------------------------ 3D volumes -- */

/* Volumes of D slices of H x W voxels, voxel (z, y, x) at z*H*W + y*W + x.
 * Adjacency 26 (the 3x3x3 cube, the 3D Moore neighbourhood) or 6 (the six
 * face neighbours); the voxel itself counts for N (reflexive), nothing
 * exists outside the volume.  These functions are separate from the 2D
 * ones above, which they leave untouched. */
static int is_offset3(int dz, int dy, int dx, int conn) {
  if (dz < -1 || dz > 1 || dy < -1 || dy > 1 || dx < -1 || dx > 1) return 0;
  if (conn == 6) return (dz != 0) + (dy != 0) + (dx != 0) <= 1;
  return 1;
}

VLO_EXPORT void vlo_near3(const uint8_t* a, int D, int H, int W, int conn,
                          uint8_t* out) {
  for (int z = 0; z < D; ++z)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        uint8_t v = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!is_offset3(dz, dy, dx, conn)) continue;
              int zz = z + dz, yy = y + dy, xx = x + dx;
              if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
              if (a[((int64_t)zz * H + yy) * W + xx]) v = 1;
            }
        out[((int64_t)z * H + y) * W + x] = v;
      }
}

/* rho phi1[phi2] in a volume, by the same BFS as vlo_reach. */
VLO_EXPORT int vlo_reach3(const uint8_t* phi1, const uint8_t* phi2, int D, int H,
                          int W, int conn, uint8_t* out) {
  int64_t n = (int64_t)D * H * W, hw = (int64_t)H * W;
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  uint8_t* pushed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!queue || !pushed) { free(queue); free(pushed); return -1; }
  int64_t head = 0, tail = 0;
  for (int64_t i = 0; i < n; ++i) {
    out[i] = phi1[i] ? 1 : 0;
    if (phi1[i]) { queue[tail++] = i; pushed[i] = 1; }
  }
  while (head < tail) {
    int64_t v = queue[head++];
    int z = (int)(v / hw), y = (int)((v % hw) / W), x = (int)(v % W);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dz == 0 && dy == 0 && dx == 0) continue;
          if (!is_offset3(dz, dy, dx, conn)) continue;
          int zz = z + dz, yy = y + dy, xx = x + dx;
          if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
          int64_t u = ((int64_t)zz * H + yy) * W + xx;
          out[u] = 1;                       /* u = pi_0, v = pi_1 */
          if (phi2[u] && !pushed[u]) {      /* u may serve as an intermediate */
            pushed[u] = 1;
            queue[tail++] = u;
          }
        }
  }
  free(queue);
  free(pushed);
  return 0;
}

/* Flood fill of a volume; label = minimum linear index of the component
 * (the first voxel met in raster order), background -1.  Returns the
 * number of components, or -1 when memory runs out. */
VLO_EXPORT int64_t vlo_ccl3(const uint8_t* m, int D, int H, int W, int conn,
                            int32_t* labels) {
  int64_t n = (int64_t)D * H * W, hw = (int64_t)H * W;
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!queue) return -1;
  for (int64_t i = 0; i < n; ++i) labels[i] = -1;
  int64_t count = 0;
  for (int64_t s = 0; s < n; ++s) {
    if (!m[s] || labels[s] != -1) continue;
    ++count;
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    labels[s] = (int32_t)s;
    while (head < tail) {
      int64_t v = queue[head++];
      int z = (int)(v / hw), y = (int)((v % hw) / W), x = (int)(v % W);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dz == 0 && dy == 0 && dx == 0) continue;
            if (!is_offset3(dz, dy, dx, conn)) continue;
            int zz = z + dz, yy = y + dy, xx = x + dx;
            if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            int64_t u = ((int64_t)zz * H + yy) * W + xx;
            if (m[u] && labels[u] == -1) {
              labels[u] = (int32_t)s;
              queue[tail++] = u;
            }
          }
    }
  }
  free(queue);
  return count;
}
