// Exact order statistic of one image channel by radix select on
// order-preserving float32 keys (three passes of 8, 12 and 12 bits; NaN
// sorts after +infinity).  The
// percentile of level q is the value of rank floor(q*(n-1)) in ascending
// order, no interpolation (the "percentiles" normalisation of Sec. 4.2).
#pragma once
#include "dev_common.cuh"

namespace vl {

struct SelectSmem {
  uint32_t hist[4096];
  uint32_t priv[EXEC_WARPS][256];  // per-warp histograms of the first digit
  uint32_t part[EXEC_THREADS];
  uint32_t digit;
  uint32_t below;
};

// One CTA selects rank k of the H x W channel `plane` (row pitch `pitch`
// elements, float or uint16 by `format`; `nc`: read-only path allowed).
// Rows go to warps and columns to lanes (coalesced); lanes of a warp that
// fall into the same bin add once (match_any), since pixels of smooth images
// crowd into a few bins of the top digits; the digit holding rank k is found
// with a block-wide scan of per-thread bin sums.  Returns the value in every
// thread (after a block barrier).
static __device__ __noinline__ float select_rank(SelectSmem& s, const void* plane, int format,
                                                 bool nc, int H, int W, int pitch, long long k) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  uint32_t prefix = 0, pmask = 0;
  unsigned long long rank = (unsigned long long)k;
  // digits of 8, 12 and 12 bits; the first digit, which every pixel hits
  // and which concentrates in a few bins, goes to per-warp histograms
  const int shifts[3] = {24, 12, 0};
  const int widths[3] = {8, 12, 12};
  for (int pass = 0; pass < 3; ++pass) {
    const int sh = shifts[pass], nb = 1 << widths[pass];
    uint32_t* hist = pass == 0 ? s.priv[warp] : s.hist;
    for (int i = tid; i < 4096; i += nthr) s.hist[i] = 0;
    if (pass == 0)
      for (int i = tid; i < EXEC_WARPS * 256; i += nthr) (&s.priv[0][0])[i] = 0;
    __syncthreads();
    constexpr int UNR = 8;  // loads in flight per lane
    for (int y = warp; y < H; y += nw) {
      const size_t row = (size_t)y * pitch;
      for (int x0 = 0; x0 < W; x0 += 32 * UNR) {
        float v[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int x = x0 + 32 * u + lane;
          v[u] = x < W ? ld_px(plane, format, nc, row + x) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          if (x0 + 32 * u >= W) break;  // uniform
          const uint32_t key = f2key(v[u]);
          const bool ok = x0 + 32 * u + lane < W && (key & pmask) == prefix;
          const uint32_t bin = (key >> sh) & (uint32_t)(nb - 1);
          const unsigned grp = __match_any_sync(0xFFFFFFFFu, ok ? bin : 0xFFFFFFFFu);
          if (ok && lane == __ffs(grp) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(grp));
        }
      }
    }
    __syncthreads();
    if (pass == 0) {
      for (int b = tid; b < 256; b += nthr) {
        uint32_t t = 0;
        for (int w = 0; w < nw; ++w) t += s.priv[w][b];
        s.hist[b] = t;
      }
      __syncthreads();
    }
    // each thread sums `per` consecutive bins; block-wide exclusive scan
    const int per = (nb + nthr - 1) / nthr;
    uint32_t sum = 0;
    for (int q = 0; q < per; ++q) {
      const int b = tid * per + q;
      if (b < nb) sum += s.hist[b];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s.part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t v = lane < nw ? s.part[lane] : 0u;
      uint32_t wi = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if (lane >= o) wi += t;
      }
      if (lane < nw) s.part[lane] = wi - v;  // exclusive sums of the warps
    }
    __syncthreads();
    const unsigned long long excl = (unsigned long long)s.part[warp] + incl - sum;
    if (sum > 0 && excl <= rank && rank < excl + sum) {  // exactly one thread
      unsigned long long acc = excl;
      for (int q = 0; q < per && tid * per + q < nb; ++q) {
        const int b = tid * per + q;
        if (acc + s.hist[b] > rank) {
          s.digit = (uint32_t)b;
          s.below = (uint32_t)acc;
          break;
        }
        acc += s.hist[b];
      }
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
