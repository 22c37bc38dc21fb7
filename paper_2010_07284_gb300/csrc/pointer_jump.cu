// Connected components by iterated pointer jumping: the paper's own GPU
// labelling (Sec. 3.3, Alg. 1), kept as an in-library comparison for the
// union-find labelling that the model checker uses.
//
// Labels are pixel indices y*W + x (the lexicographic order of (row,
// column) coordinates is the order of these indices); background is -1.
//   initialisation  -- every set pixel labels itself;
//   main iteration  -- a set pixel p whose label is q takes the largest
//                      label found in the neighbourhood of pixel q (q
//                      itself included): pointer jumping plus one step of
//                      propagation, from buffer `in` into buffer `out`;
//   reconnect       -- a set pixel p with label q, seeing a label a in its
//                      own neighbourhood larger than q's label c, raises
//                      the label of q to a (an atomic maximum: labels only
//                      grow); it repairs what the main iterations miss at
//                      concave corners;
//   termination     -- done when no set pixel has a set neighbour with a
//                      different label (a device flag read by the host).
// The host runs `period` main iterations, a reconnect, and a termination
// check per round, as the paper does (its text gives a period of 16, its
// figure captions 8).  Each round ends with one device-to-host read: the
// host-synchronised loop of the paper's design, which the persistent
// union-find executor replaces.
#include "dev_common.cuh"
#include "kernels.h"

namespace vl {

namespace {

constexpr int kPjThreads = 256;

VL_DEV bool pj_set(const uint32_t* m, int Wp, int y, int x) {
  return (__ldg(m + (size_t)y * Wp + (x >> 5)) >> (x & 31)) & 1u;
}

// Largest label in the neighbourhood of pixel (y, x), (y, x) included.
VL_DEV int32_t pj_max_around(const int32_t* lab, int H, int W, int y, int x, int conn) {
  int32_t best = -1;
  for (int dy = -1; dy <= 1; ++dy) {
    const int yy = y + dy;
    if (yy < 0 || yy >= H) continue;
    for (int dx = -1; dx <= 1; ++dx) {
      if (conn == 4 && dy != 0 && dx != 0) continue;
      const int xx = x + dx;
      if (xx < 0 || xx >= W) continue;
      best = max(best, lab[(size_t)yy * W + xx]);
    }
  }
  return best;
}

__global__ void k_pj_init(const uint32_t* __restrict__ m, int H, int W, int Wp,
                          int32_t* __restrict__ lab) {
  const long long n = (long long)H * W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / W), x = (int)(i - (long long)y * W);
    lab[i] = pj_set(m, Wp, y, x) ? (int32_t)i : -1;
  }
}

__global__ void k_pj_main(const uint32_t* __restrict__ m, int H, int W, int Wp, int conn,
                          const int32_t* __restrict__ in, int32_t* __restrict__ out) {
  const long long n = (long long)H * W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int32_t q = in[i];
    if (q < 0) { out[i] = -1; continue; }
    const int qy = q / W, qx = q - qy * W;
    out[i] = pj_max_around(in, H, W, qy, qx, conn);
  }
}

// `out` starts as a copy of `in`.
__global__ void k_pj_reconnect(int H, int W, int conn, const int32_t* __restrict__ in,
                               int32_t* out) {
  const long long n = (long long)H * W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int32_t q = in[i];
    if (q < 0) continue;
    const int y = (int)(i / W), x = (int)(i - (long long)y * W);
    const int32_t a = pj_max_around(in, H, W, y, x, conn);
    if (a > in[q]) atomicMax(out + q, a);
  }
}

// flag = 1 when some set pixel has a set neighbour with another label.
__global__ void k_pj_check(int H, int W, int conn, const int32_t* __restrict__ lab,
                           int32_t* flag) {
  const long long n = (long long)H * W;
  bool differ = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n && !differ;
       i += (long long)gridDim.x * blockDim.x) {
    const int32_t l = lab[i];
    if (l < 0) continue;
    const int y = (int)(i / W), x = (int)(i - (long long)y * W);
    for (int dy = -1; dy <= 1 && !differ; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= H) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        if (conn == 4 && dy != 0 && dx != 0) continue;
        const int xx = x + dx;
        if (xx < 0 || xx >= W) continue;
        const int32_t o = lab[(size_t)yy * W + xx];
        if (o >= 0 && o != l) { differ = true; break; }
      }
    }
  }
  if (__syncthreads_or(differ) && threadIdx.x == 0) *flag = 1;
}

int pj_grid(long long n) {
  long long b = (n + kPjThreads - 1) / kPjThreads;
  if (b > 152LL * 64) b = 152LL * 64;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t ccl_pointer_jumping(const uint32_t* mask, MaskGeom g, int conn, int period,
                                int max_rounds, int32_t* labels, int32_t* scratch,
                                int32_t* flag_dev, int32_t* flag_host, cudaStream_t st,
                                int* iterations, bool* converged) {
  const long long n = (long long)g.H * g.W;
  const int grid = pj_grid(n);
  *iterations = 0;
  *converged = false;
  int32_t* cur = labels;
  int32_t* nxt = scratch;
  k_pj_init<<<grid, kPjThreads, 0, st>>>(mask, g.H, g.W, g.Wp, cur);
  cudaError_t e = cudaGetLastError();
  for (int round = 0; !e && round < max_rounds; ++round) {
    for (int k = 0; k < period && !e; ++k) {
      k_pj_main<<<grid, kPjThreads, 0, st>>>(mask, g.H, g.W, g.Wp, conn, cur, nxt);
      e = cudaGetLastError();
      int32_t* t = cur; cur = nxt; nxt = t;
      ++*iterations;
    }
    if (e) break;
    if ((e = cudaMemcpyAsync(nxt, cur, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st))) break;
    k_pj_reconnect<<<grid, kPjThreads, 0, st>>>(g.H, g.W, conn, cur, nxt);
    if ((e = cudaGetLastError())) break;
    { int32_t* t = cur; cur = nxt; nxt = t; }
    if ((e = cudaMemsetAsync(flag_dev, 0, sizeof(int32_t), st))) break;
    k_pj_check<<<grid, kPjThreads, 0, st>>>(g.H, g.W, conn, cur, flag_dev);
    if ((e = cudaGetLastError())) break;
    if ((e = cudaMemcpyAsync(flag_host, flag_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, st))) break;
    if ((e = cudaStreamSynchronize(st))) break;
    if (*flag_host == 0) { *converged = true; break; }
  }
  if (!e && cur != labels)
    e = cudaMemcpyAsync(labels, cur, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
  if (!e) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace vl
