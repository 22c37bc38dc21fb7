// Host-side launch wrappers of the library's CUDA kernels (C++ linkage,
// internal).  Every wrapper enqueues on `st` and returns the launch error.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vl_internal.h"

namespace vl {

struct MaskGeom {
  int H, W, Wp;
  int Hs = 0;  // a volume stored as its slices stacked: rows per slice (H =
               // depth * Hs); 0 for an image
  int cth = 0; // rows of a labelling tile (even, at most CCL_TH); 0: CCL_TH
};
inline __host__ __device__ int slice_rows(const MaskGeom& g) { return g.Hs > 0 ? g.Hs : g.H; }
inline __host__ __device__ int ccl_rows(const MaskGeom& g) { return g.cth > 0 ? g.cth : CCL_TH; }

// ---- plain per-operator kernels (one launch per primitive) ----
// `plane`: one channel of H x pitch elements, float or uint16 by `format`.
cudaError_t launch_threshold(const void* plane, int format, int pitch, MaskGeom g, float t,
                             const float* t_dev, bool lt, uint32_t* out, cudaStream_t st);
cudaError_t launch_not(const uint32_t* a, MaskGeom g, uint32_t* out, cudaStream_t st);
cudaError_t launch_and(const uint32_t* a, const uint32_t* b, MaskGeom g, uint32_t* out,
                       cudaStream_t st);
cudaError_t launch_or(const uint32_t* a, const uint32_t* b, MaskGeom g, uint32_t* out,
                      cudaStream_t st);
cudaError_t launch_andnot(const uint32_t* a, const uint32_t* b, MaskGeom g, uint32_t* out,
                          cudaStream_t st);
cudaError_t launch_const(MaskGeom g, bool value, uint32_t* out, cudaStream_t st);
cudaError_t launch_near(const uint32_t* a, MaskGeom g, int conn, uint32_t* out,
                        cudaStream_t st);
cudaError_t launch_select(const void* plane, int format, int pitch, int H, int W, long long rank,
                          float* out, cudaStream_t st);
// The same over the whole grid, for large channels; scratch: device memory
// of select_wide_scratch_bytes() (reused call after call on one stream).
size_t select_wide_scratch_bytes();
cudaError_t launch_select_wide(const void* plane, int format, int pitch, int H, int W,
                               long long rank, float* out, void* scratch, cudaStream_t st);
// out = a (op) b per pixel (op an ArithOp, A_ADD .. A_DIV); b null: the
// constant c.
cudaError_t launch_arith(int op, const void* a, int a_format, const void* b, int b_format, float c,
                         float* out, int H, int W, int pitch, cudaStream_t st);

// ---- connected components (tile-local, merge, flags, final) ----
struct CclScratch {
  int32_t* G;       // union-find: H*W int32 for labels (the label array
                    // itself), 2*H*W for rho (pixel ids, then the keys of
                    // unseeded components)
  int32_t tile_cap; // per-tile capacity of tpar / tflag (ccl_tile_cap_host)
  int32_t* tpar;    // tiles * tile_cap int32: saved tile union-find state
  uint8_t* tflag;   // tiles * tile_cap bytes: saved tile flags
};
// Labelling tiles: rows over all slices (Hs 0: an image; cth: rows per
// tile, even, at most CCL_TH), columns, per-tile saved-state capacity.
int ccl_tiles_y(int H, int Hs = 0, int cth = CCL_TH);
int ccl_tiles_x(int Wp);
int ccl_tile_cap_host(int Wp, int cth = CCL_TH);
// Border merge units (one warp each): words of horizontal tile borders and
// 32-row pieces of vertical ones.
long long ccl_merge_units(int H, int Wp, int Hs = 0, int cth = CCL_TH);
size_t ccl_smem_bytes();
// Set the labelling kernels' shared-memory attribute on the current device
// (done by every labelling launch; call it before a stream capture).
cudaError_t ccl_configure();

// Labels: sc.G is the labels array itself (it doubles as the union-find).
// Tiles of ccl_rows(g) rows: sc.tpar / sc.tflag hold ccl_tiles_y(H, Hs,
// ccl_rows(g)) * ccl_tiles_x(Wp) tiles of ccl_tile_cap_host(Wp, ccl_rows(g)).
// The same for launch_rz.
cudaError_t launch_ccl_labels(const uint32_t* mask, MaskGeom g, int conn, CclScratch sc,
                              int32_t* status, cudaStream_t st);
// Component select Z (rho core): Z = phi2-components meeting N phi1.
cudaError_t launch_rz(const uint32_t* phi1, const uint32_t* phi2, MaskGeom g, int conn,
                      CclScratch sc, uint32_t* Z, int32_t* status, cudaStream_t st);

// ---- volumes (D slices of Hs rows stacked; g.Hs set) ----
// conn: 26 (cube) or 6 (faces).
cudaError_t launch_near3(const uint32_t* a, MaskGeom g, int conn, uint32_t* out, cudaStream_t st);
// Full labels: sc.G is the labels array; sc.tpar / sc.tflag sized for
// ccl_tiles_y(H, Hs) * ccl_tiles_x(Wp) tiles.
cudaError_t launch_labels3(const uint32_t* mask, MaskGeom g, int conn, CclScratch sc,
                           int32_t* status, cudaStream_t st);
struct Rz3Scratch {
  CclScratch ccl;   // G: H*W int32 labels of phi2
  uint8_t* F;       // H*W bytes: flag per component root
  uint32_t* seed;   // H x Wp words
};
cudaError_t launch_rz3(const uint32_t* phi1, const uint32_t* phi2, MaskGeom g, int conn,
                       Rz3Scratch sc, uint32_t* Z, int32_t* status, cudaStream_t st);

// ---- mask conversion ----
cudaError_t launch_pack_u8(const uint8_t* src, MaskGeom g, uint32_t* out, cudaStream_t st);
cudaError_t launch_unpack_u8(const uint32_t* src, MaskGeom g, uint8_t* out, cudaStream_t st);
cudaError_t launch_clear_padding(uint32_t* m, MaskGeom g, cudaStream_t st);

// ---- the paper's pointer-jumping labelling (comparison only) ----
// Runs rounds of `period` main iterations + reconnect + termination check
// until converged or `max_rounds`; synchronises `st` once per round.
// labels / scratch: H*W int32 each; flag_dev: one int32; flag_host: host.
cudaError_t ccl_pointer_jumping(const uint32_t* mask, MaskGeom g, int conn, int period,
                                int max_rounds, int32_t* labels, int32_t* scratch,
                                int32_t* flag_dev, int32_t* flag_host, cudaStream_t st,
                                int* iterations, bool* converged);

// ---- persistent executor ----
struct ExecLaunch {
  const DevJob* jobs;
  const WorkItem* items;
  int32_t n_items;
  int32_t* head;           // work-queue head (zeroed before launch)
  int32_t* done;           // per (job, step) finished sub-items (zeroed)
  const int32_t* need;     // per (job, step) sub-items in total
  int64_t spin_limit;
  int32_t group_buffers;   // shared-memory buffers per group tile
  int32_t group_bh;        // rows per buffer (gth + 2*HMAX)
  int32_t group_bw;        // words per buffer (gtww + 2)
  int32_t grid;            // CTAs
  int32_t smem_bytes;      // dynamic shared memory per CTA (groups stage rank
                           // planes in what their buffers leave free)
  unsigned long long* trace;  // optional: per (job, step) {start, end, busy, wait} in ns
};
size_t exec_smem_bytes(int group_buffers, int group_bh, int group_bw);
cudaError_t exec_configure(size_t smem_bytes, int* max_ctas_per_sm);
cudaError_t launch_exec(const ExecLaunch& L, cudaStream_t st);

}  // namespace vl
