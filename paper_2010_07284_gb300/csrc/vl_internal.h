// Internal data structures shared by the host compiler/runtime and the CUDA
// kernels.  Plain structs only (no STL) so that device code can read them.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define VL_HD_INLINE __host__ __device__ __forceinline__
#else
#define VL_HD_INLINE inline
#endif

namespace vl {

// ----------------------------------------------------------------- geometry
// Bit-packed masks: Wp = 4 * ceil(W / 128) words per row, LSB first.
static inline int words_per_row(int w) { return ((w + 127) / 128) * 4; }

// Connected-component tiles: up to CCL_TH rows x CCL_TWW words (1024 px),
// labelled as CCL_NS strips of two rows; one lane owns a 32-px word.
constexpr int CCL_TH = 32;
constexpr int CCL_TWW = 32;
constexpr int CCL_NS = CCL_TH / 2;
// A strip run can start at every column under 4-adjacency (checkerboard).
constexpr int CCL_MAXRUNS = CCL_NS * CCL_TWW * 32;

constexpr int EXEC_THREADS = 512;  // threads per CTA of every tiled kernel
constexpr int EXEC_WARPS = EXEC_THREADS / 32;

// Device status word values (match vl_status where they overlap).
constexpr int ST_OK = 0;
constexpr int ST_TIMEOUT = 6;
constexpr int ST_INTERNAL = 8;
// Which consistency check failed (bits 8.. of the status word, with
// ST_INTERNAL in the low byte).
constexpr int RS_GFIND = 1 << 8;     // global find ran past its bound
constexpr int RS_GUNION = 2 << 8;    // global union ran past its bound
constexpr int RS_FLIST = 3 << 8;     // (unused: no flagged-root list any more)
constexpr int RS_TLOAD = 4 << 8;     // saved tile state out of range
constexpr int RS_TRUNS = 5 << 8;     // more strip runs than a tile holds
constexpr int RS_SUNION = 6 << 8;    // shared union-find ran past its bound
constexpr int RS_GRANGE = 7 << 8;    // global union-find entry outside the image

// --------------------------------------------------------- group bytecode
// One instruction of a fused tile group.  Buffers are shared-memory tiles
// of (th + 2*halo) rows x (tww + 2) words; `h` is the halo (in rows and
// pixels) over which this node's value is needed.
enum InsnOp : uint8_t {
  I_NOP = 0,
  I_THR = 1,     // dst = image[img].channel[ch] (> or <) t      (aux bit0: lt,
                 //   bit1: t comes from the job's percentile slot `slot`)
  I_LOAD = 2,    // dst = materialised mask slot `slot`
  I_NOT = 3,     // dst = not a
  I_AND = 4,     // dst = a and b
  I_OR = 5,      // dst = a or b
  I_NEAR = 6,    // dst = N a (connectivity of the formula)
  I_CONST = 7,   // dst = all-false (aux 0) or all-true (aux 1)
  I_STORE = 8,   // materialised mask slot `slot` = a   (core region only)
  I_ANDNOT = 9,  // dst = a and not b
  I_RTHR = 10,   // dst = threshold by rank code: table a, code bound K = img
                 //   (as uint16), code bits = ch, first plane = slot; aux
                 //   bit0: lt (see RankTab)
};

// Bit of Insn::op: a block barrier precedes the instruction (the compiler
// places one only where a thread may touch a buffer word that another
// thread touched since the previous barrier).
constexpr uint8_t I_SYNC = 0x80;

struct Insn {        // 16 bytes
  uint8_t op;        // InsnOp, with I_SYNC
  uint8_t dst;
  uint8_t a;
  uint8_t b;
  int16_t h;         // halo of this node within the group
  int16_t slot;      // materialised-mask slot / percentile slot
  int16_t img;       // image index (THR)
  int16_t ch;        // channel (THR)
  float t;           // threshold constant (THR)
};
static_assert(sizeof(Insn) == 16, "Insn layout");
VL_HD_INLINE int insn_op(const Insn& in) { return in.op & ~I_SYNC; }

// -------------------------------------------------------------- plan steps
enum StepKind : int32_t {
  SK_PCT = 0,        // percentile selects: one item per percentile slot
  SK_GROUP = 1,      // fused pointwise/N tile group: one item per tile
  SK_RZ_LOCAL = 2,   // rho batch, tile-local labelling + publish: item = (rz, tile)
  SK_RZ_MERGE = 3,   // rho batch, union across tile borders: item = (rz, chunk)
  SK_RZ_UNUSED = 4,  // (no longer emitted: the seed flag travels with the keys)
  SK_RZ_FINAL = 5,   // rho batch, relabel + write Z: item = (rz, tile)
  SK_RANK = 6,       // rank codes of threshold tables: item = (table, row block)
  SK_ARITH = 7,      // number terms: item = row block, writes the number images
};

// Rows of one arithmetic work item.
constexpr int ARITH_ROWS = 8;

// Number terms of a formula as one straight-line program run per pixel on a
// register file of floats: A_VALUE loads image[img].channel[ch], the
// operations read registers a and b (b = kArithConst: the constant c) and
// write dst, A_STORE writes register a to number image `img` (counted from
// the first number image).  Every operation rounds to float once.
enum ArithOp : uint8_t { A_VALUE = 0, A_ADD = 1, A_SUB = 2, A_MUL = 3, A_DIV = 4, A_STORE = 5 };
constexpr uint8_t kArithConst = 0xFF;
constexpr int kArithMaxRegs = 16;
constexpr int kArithMaxInsns = 1024;
struct ArithInsn {   // 12 bytes
  uint8_t op, dst, a, b;
  int16_t img, ch;
  float c;
};
static_assert(sizeof(ArithInsn) == 12, "ArithInsn layout");

// Rows of one rank-code work item.
constexpr int RANK_ROWS = 8;

struct StepDesc {
  int32_t kind;
  int32_t insn_off;  // groups: first instruction (into the formula's insns)
  int32_t insn_cnt;
  int32_t halo;      // groups: halo rows/px
  int32_t rz_off;    // rho batches: first RZ entry
  int32_t rz_cnt;
  int32_t pct_off;   // percentile step: first PCT entry
  int32_t pct_cnt;
  int32_t rank_mask; // groups: rank tables (< 32) its I_RTHR read, one bit each
  int32_t rank_halo; // groups: largest halo of those I_RTHR
  int32_t n_bufs;    // groups: tile buffers its instructions use (0 .. n_bufs-1);
                     //   the shared-memory stage of rank planes follows them
};

// Rank codes of one image channel against the sorted distinct constant
// thresholds t_1 < ... < t_m of a formula on that channel: a pixel value v
// has code c = 2 * #{k : t_k < v} + [v equals some t_k] (0 for NaN), kept
// as `nbits` bit planes (bit b of every pixel's code in plane plane0 + b)
// plus a plane of NaN pixels (plane0 + nbits).  Then v > t_k exactly when
// c >= 2k, and v < t_k exactly when c < 2k - 1 and v is not NaN, so every
// threshold of the table becomes one bit-sliced comparison with a constant.
struct RankTab {
  int32_t img, ch;
  int32_t m;         // thresholds in the table
  int32_t nbits;     // code bits: bit length of 2m + 1
  int32_t val_off;   // first threshold value in the formula's value array
  int32_t plane0;    // first plane of the table in the job's plane array
};

// Component select Z = union of phi2-components meeting N phi1 (the core of
// rho, Sec. 3.2); the compiler lowers rho phi1[phi2] to N(phi1 or Z).
struct RzDesc {
  int16_t phi1_slot;
  int16_t phi2_slot;
  int16_t z_slot;
  int16_t scratch;   // index of the job's CCL scratch set used
};

struct PctDesc {
  int16_t img;
  int16_t ch;
  int16_t slot;      // percentile slot written
  int16_t pad;
  double q;
};

// ----------------------------------------------------- executor job table
// Pixel formats of number images.
constexpr int32_t PX_F32 = 0;
constexpr int32_t PX_U16 = 1;

struct DevImage {
  const void* data;        // number images: channels planes of H x pitch
                           //   elements (float, or uint16 by `format`)
  const uint32_t* mask;    // mask images: H x Wp words
  int32_t channels;
  int32_t is_mask;
  int32_t format;          // PX_F32 or PX_U16
  int32_t written;         // 1: written earlier in the same launch (number
                           //   images of SK_ARITH): read through L2, not the
                           //   read-only path
};

struct DevJob {
  int32_t H, W, Wp, pitch;      // pitch in floats = 32 * Wp
  int32_t n_steps;
  int32_t step_base;            // into the launch's step table
  int32_t gth, gtww;            // group tile rows / words
  int32_t g_tiles_y, g_tiles_x; // group tiles
  int32_t c_tiles_y, c_tiles_x; // CCL tiles
  int32_t conn;
  int32_t n_images;
  const DevImage* images;
  uint32_t* const* slots;       // materialised mask slots
  const Insn* insns;
  const StepDesc* steps;        // this job's formula steps
  const int32_t* dep_off;       // step dependencies (CSR, job-relative steps)
  const int32_t* deps;
  const RzDesc* rz;
  const PctDesc* pct;
  float* pct_val;               // percentile values by slot
  // CCL scratch sets, one per select of a batch step, `set_bytes` apart:
  // union-find over keys (G, 2 * H * W entries: pixel ids and the keys of
  // unseeded components), saved tile union-find state and flags (tiles x
  // tile_cap)
  unsigned char* rzs;
  int64_t set_bytes;
  int64_t off_tpar, off_tflag;
  int32_t tile_cap;
  int32_t c_th;                 // rows of a labelling tile (16 or 32)
  int32_t* status;              // device status word of this job
  const RankTab* rtab;          // rank tables of the formula
  const float* rvals;           //   their sorted threshold values
  int32_t n_rtab;
  int32_t pad_;
  uint32_t* planes;             // rank-code planes, H x Wp words each
  const ArithInsn* arith;       // number-term program (SK_ARITH)
  int32_t n_arith;
  int32_t first_num_image;      // image index of number image 0
};

VL_HD_INLINE int32_t* rz_G(const DevJob& J, int k) {
  return reinterpret_cast<int32_t*>(J.rzs + k * J.set_bytes);
}
VL_HD_INLINE int32_t* rz_tpar(const DevJob& J, int k) {
  return reinterpret_cast<int32_t*>(J.rzs + k * J.set_bytes + J.off_tpar);
}
VL_HD_INLINE uint8_t* rz_tflag(const DevJob& J, int k) { return J.rzs + k * J.set_bytes + J.off_tflag; }

// One work item of the persistent executor: a range of `count` consecutive
// sub-items (tiles, chunks, rz x tile) of one step of one job.
struct WorkItem {
  int32_t job;
  int32_t step;        // step index within the job
  int32_t first;       // first sub-item
  int32_t count;       // sub-items in this item
};

}  // namespace vl
