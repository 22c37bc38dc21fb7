// Exact order statistic of one image channel by radix select on
// order-preserving float32 keys (three passes of 11, 11 and 10 bits).  The
// percentile of level q is the value of rank floor(q*(n-1)) in ascending
// order, no interpolation (the "percentiles" normalisation of Sec. 4.2).
#pragma once
#include "dev_common.cuh"

namespace vl {

struct SelectSmem {
  uint32_t hist[2048];
  uint32_t part[EXEC_THREADS];
  uint32_t digit;
  uint32_t below;
};

// One CTA selects rank k of the H x W channel `plane` (row pitch `pitch`).
// Returns the value in every thread (after a block barrier).
VL_DEV float select_rank(SelectSmem& s, const float* plane, int H, int W, int pitch,
                         long long k) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  uint32_t prefix = 0, pmask = 0;
  unsigned long long rank = (unsigned long long)k;
  const int shifts[3] = {21, 10, 0};
  const int widths[3] = {11, 11, 10};
  for (int pass = 0; pass < 3; ++pass) {
    const int sh = shifts[pass], nb = 1 << widths[pass];
    for (int i = tid; i < 2048; i += nthr) s.hist[i] = 0;
    __syncthreads();
    const long long n = (long long)H * pitch;
    for (long long i = tid; i < n; i += nthr) {
      int x = (int)(i % pitch);
      if (x >= W) continue;
      uint32_t key = f2key(__ldg(plane + i));
      if ((key & pmask) == prefix) atomicAdd(&s.hist[(key >> sh) & (nb - 1)], 1u);
    }
    __syncthreads();
    // bins per thread, then an exclusive scan of the partial sums
    const int per = (nb + nthr - 1) / nthr;
    uint32_t sum = 0;
    for (int q = 0; q < per; ++q) {
      int bidx = tid * per + q;
      if (bidx < nb) sum += s.hist[bidx];
    }
    s.part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
      unsigned long long acc = 0;
      int t = 0;
      for (; t < nthr; ++t) {
        if (acc + s.part[t] > rank) break;
        acc += s.part[t];
      }
      int d = t * per;
      for (; d < nb; ++d) {
        if (acc + s.hist[d] > rank) break;
        acc += s.hist[d];
      }
      s.digit = (uint32_t)min(d, nb - 1);
      s.below = (uint32_t)acc;
    }
    __syncthreads();
    rank -= s.below;
    prefix |= s.digit << sh;
    pmask |= (uint32_t)(nb - 1) << sh;
    __syncthreads();
  }
  return key2f(prefix);
}

}  // namespace vl
