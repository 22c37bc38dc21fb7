// Persistent batched executor.
//
// One launch walks a device work list.  An item is a range of sub-items
// (tiles, merge chunks, selects) of one step of one job; items are ordered
// so that everything an item depends on comes earlier in the list.  CTAs pop
// items with an atomic counter, so an item's dependencies were popped by
// CTAs already running: the earliest unfinished item can always progress,
// and the launch needs no co-residency guarantee.  Before running, an item
// waits (bounded, with back-off) until every sub-item of each step its
// step depends on is done; a wait that runs out records VL_ERR_TIMEOUT in the job's
// status word and the job's remaining items are skipped.  This replaces the
// paper's host-side event chaining and host-checked CCL termination
// (Sec. 3.2-3.3) with device-side counters: the host never waits.
#include "dev_ccl.cuh"
#include "dev_common.cuh"
#include "dev_group.cuh"
#include "dev_select.cuh"
#include "kernels.h"

namespace vl {

namespace {

VL_DEV unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

VL_DEV int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Rank codes of rows [y0, y1) of one channel against the sorted table tv
// (see RankTab): one warp per 32-pixel word, one lane per pixel; code bit b
// of the word's pixels is a ballot, written to plane b (lane b writes it).
// A warp takes RANK_UNR words at a time: their loads are in flight
// together, and their searches (branch-free, the same number of steps for
// every lane) interleave.
constexpr int RANK_UNR = 4;
VL_DEV void rank_rows(const float* tv, const RankTab& T, const void* plane, int format, bool nc,
                      int H, int W, int Wp, int pitch, int y0, int y1, uint32_t* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t pstride = (size_t)H * Wp;
  const int nwords = (y1 - y0) * Wp;
  for (int base = warp * RANK_UNR; base < nwords; base += nw * RANK_UNR) {
    float v[RANK_UNR];
    bool in[RANK_UNR];
#pragma unroll
    for (int u = 0; u < RANK_UNR; ++u) {
      const int idx = base + u;
      const int y = y0 + idx / Wp, w = idx - (idx / Wp) * Wp;
      const int x = 32 * w + lane;
      in[u] = idx < nwords && x < W;
      v[u] = 0.f;
      if (in[u]) {
        const size_t i = (size_t)y * pitch + x;
        if (format == PX_U16) v[u] = (float)static_cast<const unsigned short*>(plane)[i];
        else v[u] = nc ? __ldg(static_cast<const float*>(plane) + i) : __ldcg(static_cast<const float*>(plane) + i);
      }
    }
    // lower bound: the number of table values below v (none for NaN)
    int lo[RANK_UNR];
#pragma unroll
    for (int u = 0; u < RANK_UNR; ++u) lo[u] = 0;
    for (int n = T.m; n > 1;) {
      const int half = n >> 1;
#pragma unroll
      for (int u = 0; u < RANK_UNR; ++u) lo[u] = tv[lo[u] + half - 1] < v[u] ? lo[u] + half : lo[u];
      n -= half;
    }
#pragma unroll
    for (int u = 0; u < RANK_UNR; ++u) {
      const int idx = base + u;
      if (idx >= nwords) break;  // uniform: idx is the same for the warp
      if (T.m > 0 && tv[lo[u]] < v[u]) ++lo[u];
      const unsigned code = 2u * (unsigned)lo[u] + ((lo[u] < T.m && tv[lo[u]] == v[u]) ? 1u : 0u);
      uint32_t mine = 0;
      for (int b = 0; b < T.nbits; ++b) {
        const uint32_t word = __ballot_sync(FULL, in[u] && ((code >> b) & 1u));
        if (lane == b) mine = word;
      }
      const uint32_t nan = __ballot_sync(FULL, in[u] && v[u] != v[u]);
      if (lane == T.nbits) mine = nan;
      const int y = y0 + idx / Wp, w = idx - (idx / Wp) * Wp;
      if (lane <= T.nbits) out[(size_t)lane * pstride + (size_t)y * Wp + w] = mine;
    }
  }
}

// Number terms of rows [sub * ARITH_ROWS, +ARITH_ROWS): the program runs per
// pixel on a register file in shared memory (register q of thread t at
// R[q * blockDim + t]; no local memory).
VL_DEV void arith_rows(const DevJob& J, int sub, unsigned char* smem) {
  const int nt = blockDim.x, n = J.n_arith;
  float* R = reinterpret_cast<float*>(smem);
  ArithInsn* prog = reinterpret_cast<ArithInsn*>(R + (size_t)kArithMaxRegs * nt);
  for (int i = threadIdx.x; i < n; i += nt) prog[i] = J.arith[i];
  __syncthreads();
  float* r = R + threadIdx.x;
  const size_t plane = (size_t)J.H * J.pitch;
  const int y0 = sub * ARITH_ROWS, rows = min(J.H - y0, ARITH_ROWS);
  for (int idx = threadIdx.x; idx < rows * J.W; idx += nt) {
    const int y = y0 + idx / J.W, x = idx - (idx / J.W) * J.W;
    const size_t off = (size_t)y * J.pitch + x;
    for (int k = 0; k < n; ++k) {
      const ArithInsn A = prog[k];
      if (A.op == A_VALUE) {
        const DevImage im = J.images[A.img];
        r[A.dst * nt] = ld_px(chan_ptr(im, A.ch, plane), im.format, !im.written, off);
      } else if (A.op == A_STORE) {
        float* out = static_cast<float*>(const_cast<void*>(J.images[J.first_num_image + A.img].data));
        out[off] = r[A.a * nt];
      } else {
        const float u = r[A.a * nt];
        const float w = A.b == kArithConst ? A.c : r[A.b * nt];
        // one IEEE rounding per operation: the _rn intrinsics are never
        // contracted into fused multiply-adds
        float z;
        switch (A.op) {
          case A_ADD: z = __fadd_rn(u, w); break;
          case A_SUB: z = __fsub_rn(u, w); break;
          case A_MUL: z = __fmul_rn(u, w); break;
          default: z = __fdiv_rn(u, w); break;
        }
        r[A.dst * nt] = z;
      }
    }
  }
}

VL_DEV void run_subitem(const DevJob& J, const StepDesc& S, int sub, int per_rz,
                        unsigned char* smem, const ExecLaunch& L) {
  const int npx = J.H * J.W;
  switch (S.kind) {
    case SK_PCT: {
      SelectSmem& s = *reinterpret_cast<SelectSmem*>(smem);
      const PctDesc d = J.pct[S.pct_off + sub];
      const DevImage im = J.images[d.img];
      const long long n = (long long)J.H * J.W;
      const long long rank = (long long)(d.q * (double)(n - 1));
      const float v = select_rank(s, chan_ptr(im, d.ch, (size_t)J.H * J.pitch), im.format,
                                  !im.written, J.H, J.W, J.pitch, rank);
      if (threadIdx.x == 0) J.pct_val[d.slot] = v;
      break;
    }
    case SK_GROUP: {
      GroupCtx c;
      c.H = J.H; c.W = J.W; c.Wp = J.Wp; c.pitch = J.pitch;
      const int ty = sub / J.g_tiles_x, tx = sub - ty * J.g_tiles_x;
      c.r0 = ty * J.gth; c.w0 = tx * J.gtww;
      c.th = min(J.gth, J.H - c.r0); c.tww = min(J.gtww, J.Wp - c.w0);
      c.halo = S.halo;
      c.bh = L.group_bh; c.bw = L.group_bw;
      c.conn = J.conn;
      c.buf = reinterpret_cast<uint32_t*>(smem);
      c.images = J.images; c.slots = J.slots; c.pct_val = J.pct_val;
      c.rtab = J.rtab; c.planes = J.planes; c.pstride = (size_t)J.H * J.Wp;
      // the stage of rank planes follows the buffers this group uses
      const int nbuf = min(max(S.n_bufs, 1), L.group_buffers);
      c.stage = c.buf + (size_t)nbuf * c.bh * c.bw;
      c.stage_cap = L.smem_bytes / 4 - nbuf * c.bh * c.bw;
      c.rank_mask = S.rank_mask; c.rank_halo = S.rank_halo;
      group_tile(c, J.insns + S.insn_off, S.insn_cnt);
      break;
    }
    case SK_RANK: {
      const int per_tab = (J.H + RANK_ROWS - 1) / RANK_ROWS;
      const int tab = sub / per_tab, rb = sub - tab * per_tab;
      const RankTab T = J.rtab[tab];
      float* tv = reinterpret_cast<float*>(smem);
      for (int i = threadIdx.x; i < T.m; i += blockDim.x) tv[i] = J.rvals[T.val_off + i];
      __syncthreads();
      const DevImage im = J.images[T.img];
      rank_rows(tv, T, chan_ptr(im, T.ch, (size_t)J.H * J.pitch), im.format, !im.written, J.H,
                J.W, J.Wp, J.pitch, rb * RANK_ROWS, min(J.H, (rb + 1) * RANK_ROWS),
                J.planes + (size_t)T.plane0 * J.H * J.Wp);
      break;
    }
    case SK_ARITH:
      arith_rows(J, sub, smem);
      break;
    case SK_RZ_LOCAL:
    case SK_RZ_FINAL: {
      CclSmem& s = *reinterpret_cast<CclSmem*>(smem);
      const int j = sub / per_rz, tile = sub - j * per_rz;
      const RzDesc r = J.rz[S.rz_off + j];
      const int k = r.scratch;
      const CclGeom geo = ccl_geom(J.H, J.W, J.Wp, tile, J.c_tiles_x, J.H, J.c_th);
      const uint32_t* phi1 = J.slots[r.phi1_slot];
      const uint32_t* phi2 = J.slots[r.phi2_slot];
      int32_t* tpar = rz_tpar(J, k) + (size_t)tile * J.tile_cap;
      uint8_t* tflag = rz_tflag(J, k) + (size_t)tile * J.tile_cap;
      if (S.kind == SK_RZ_LOCAL) {
        if (!ccl_tile_label(s, phi2, phi1, geo, J.conn, false, J.status)) break;
        ccl_encode_roots(s, geo, ENC_PUBLISH_RZ, rz_G(J, k), 2 * npx, npx, J.status);
        ccl_publish_border(s, geo, rz_G(J, k));
        ccl_tile_save(s, tpar, tflag);
      } else {
        if (!ccl_tile_load(s, phi2, geo, J.conn, tpar, tflag, J.status)) break;
        ccl_encode_roots(s, geo, ENC_SELECT, rz_G(J, k), 2 * npx, npx, J.status);
        ccl_write_select(s, geo, J.slots[r.z_slot]);
      }
      break;
    }
    case SK_RZ_MERGE: {
      const int j = sub / per_rz, chunk = sub - j * per_rz;
      const RzDesc r = J.rz[S.rz_off + j];
      const int n = merge_units(J.H, J.Wp, J.c_tiles_x, J.H, J.c_th);
      const int nw = blockDim.x >> 5;
      for (int u = chunk * nw + (threadIdx.x >> 5); u < n; u += per_rz * nw)
        ccl_merge_unit(J.slots[r.phi2_slot], J.H, J.W, J.Wp, u, J.conn, rz_G(J, r.scratch),
                       2 * npx, J.status, J.H, J.c_th);
      break;
    }
    default:
      break;
  }
}

__global__ void __launch_bounds__(EXEC_THREADS, 2) k_exec(ExecLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item, s_skip;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(L.head, 1);
    __syncthreads();
    const int idx = s_item;
    if (idx >= L.n_items) break;
    const WorkItem it = L.items[idx];
    const DevJob& J = L.jobs[it.job];
    const StepDesc S = J.steps[it.step];
    const int ci = J.step_base + it.step;
    unsigned long long t_pop = 0, t_go = 0;
    if (threadIdx.x == 0) {
      if (L.trace) t_pop = now_ns();
      int skip = 0;
      const int d0 = J.dep_off[it.step], d1 = J.dep_off[it.step + 1];
      // a negative limit makes every wait expire at once (tests of the
      // timeout path); otherwise poll with back-off up to the limit
      if (d1 > d0 && L.spin_limit < 0) {
        set_status(J.status, ST_TIMEOUT);
        skip = 1;
      }
      for (int q = d0; q < d1 && !skip; ++q) {
        const int dep = J.step_base + J.deps[q];
        const int32_t* ctr = L.done + dep;
        const int need = L.need[dep];
        long long spins = 0;
        unsigned ns = 32;
        while (ld_acquire(ctr) < need) {
          if (++spins > L.spin_limit) {
            set_status(J.status, ST_TIMEOUT);
            skip = 1;
            break;
          }
          __nanosleep(ns);
          if (ns < 1024) ns <<= 1;
        }
      }
      if (ldcg(J.status) != 0) skip = 1;
      s_skip = skip;
      if (L.trace) t_go = now_ns();
    }
    __syncthreads();
    if (!s_skip) {
      int per_rz = 1;
      if (S.kind == SK_RZ_LOCAL || S.kind == SK_RZ_MERGE || S.kind == SK_RZ_FINAL)
        per_rz = L.need[ci] / S.rz_cnt;
      for (int k = 0; k < it.count; ++k) {
        run_subitem(J, S, it.first + k, per_rz, smem_raw, L);
        __syncthreads();
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(L.done + ci, it.count);
      if (L.trace) {
        const unsigned long long t_end = now_ns();
        unsigned long long* tr = L.trace + 4 * (size_t)ci;
        atomicMin(tr + 0, t_go);
        atomicMax(tr + 1, t_end);
        atomicAdd(tr + 2, t_end - t_go);
        atomicAdd(tr + 3, t_go - t_pop);
      }
    }
  }
}

}  // namespace

size_t exec_smem_bytes(int group_buffers, int group_bh, int group_bw) {
  size_t g = (size_t)group_buffers * group_bh * group_bw * 4;
  size_t m = sizeof(CclSmem);
  if (sizeof(SelectSmem) > m) m = sizeof(SelectSmem);
  const size_t arith = (size_t)kArithMaxRegs * EXEC_THREADS * 4 + sizeof(ArithInsn) * kArithMaxInsns;
  if (arith > m) m = arith;
  if (g > m) m = g;
  return (m + 15) & ~(size_t)15;
}

cudaError_t exec_configure(size_t smem_bytes, int* max_ctas_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_exec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_ctas_per_sm, k_exec, EXEC_THREADS,
                                                       smem_bytes);
}

cudaError_t launch_exec(const ExecLaunch& L, cudaStream_t st) {
  k_exec<<<L.grid, EXEC_THREADS, (size_t)L.smem_bytes, st>>>(L);
  return cudaGetLastError();
}

}  // namespace vl
