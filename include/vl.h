/*
 * vl.h -- C ABI of a GB300-native (sm_103a) spatial model checker for the
 * logic SLCS on 2D images.
 *
 * What it computes (paper "A spatial model checker in GPU", Sec. 2): a
 * formula phi ::= p | not phi | phi1 and phi2 | N phi | rho phi1[phi2]
 * (Eq. (1) of Sec. 2) is interpreted on the pixels of an image of fixed size,
 * and its value is the binary image of the pixels satisfying it.  Atomic
 * propositions are thresholds on an image feature; not / and are pixel-wise;
 * N phi is the dilation of phi by the Moore neighbourhood (8-adjacency) or by
 * the cross (4-adjacency); rho phi1[phi2] holds at x when some path from x
 * reaches a phi1 pixel with every intermediate pixel in phi2.  As in the
 * paper's tool (Sec. 3.2), a formula is a DAG of operator tasks whose
 * sub-expressions are shared, evaluated on data that stays on the device
 * (Sec. 3.2) and read back only on request; rho reduces to connected
 * component labelling (Sec. 3.2-3.3).
 *
 * Conventions for every entry point:
 *  - Return value: a vl_status.  Nothing aborts or throws across the ABI.
 *    After an error, vl_last_error(ctx) gives a one-line message.
 *  - Handles (vl_context, vl_image, vl_formula, vl_result, vl_server) are
 *    owned by the library; release each with vl_free().  vl_free(NULL) is a
 *    no-op.  A handle must not be freed while work that uses it is still
 *    queued on a stream (call vl_result_sync first).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Work is enqueued asynchronously and ordered on that
 *    stream like any CUDA call; the host does not wait unless an entry point
 *    says so.
 *  - Pointers: "host" pointers are ordinary CPU memory (pinned or not);
 *    "device" pointers are CUDA global memory on the context's device.
 *  - Masks are bit-packed, LSB first: pixel (y, x) of an H x W mask is bit
 *    (x mod 32) of word y*Wp + x/32, with Wp = 4 * ceil(W / 128) words per
 *    row (rows padded to 16 bytes).  Padding bits are always 0.
 *  - Labels are int32, row-major H x W; a component is labelled by its
 *    minimum linear index y*W + x; background pixels are -1.
 */
#ifndef VL_H_
#define VL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(_WIN32)
#define VL_API __declspec(dllexport)
#else
#define VL_API __attribute__((visibility("default")))
#endif

/* ------------------------------------------------------------------ status */

typedef enum {
  VL_OK = 0,
  VL_ERR_ARG = 1,       /* bad argument (null pointer, bad size, bad handle) */
  VL_ERR_FORMULA = 2,   /* malformed formula: operand order, arity, op code */
  VL_ERR_SHAPE = 3,     /* images of a call do not share H x W, bad channel */
  VL_ERR_OOM = 4,       /* device memory could not be obtained */
  VL_ERR_CUDA = 5,      /* a CUDA runtime call failed */
  VL_ERR_TIMEOUT = 6,   /* a bounded device-side wait ran out (status word) */
  VL_ERR_BUSY = 7,      /* not finished yet / queue full */
  VL_ERR_INTERNAL = 8,  /* a device-side consistency check failed */
  VL_ERR_CANCELLED = 9  /* a served query was cancelled */
} vl_status;

/* ----------------------------------------------------------------- handles */

typedef struct vl_context vl_context;
typedef struct vl_image vl_image;
typedef struct vl_formula vl_formula;
typedef struct vl_result vl_result;
typedef struct vl_server vl_server;

/* Execution forms. */
typedef enum {
  VL_EXEC_FUSED = 0,  /* persistent executor: fused tile groups, one launch */
  VL_EXEC_PLAIN = 1   /* one kernel launch per primitive operator */
} vl_exec_mode;

typedef struct {
  int32_t device;         /* CUDA device ordinal (default 0) */
  int32_t exec_mode;      /* vl_exec_mode for vl_eval (default FUSED) */
  int32_t use_graphs;     /* capture batched launches in CUDA graphs (1) */
  int32_t trace;          /* record a device-side step timeline in batched
                             launches (see vl_batch_trace); default 0 */
  int64_t spin_limit;     /* cap on polls of every device-side wait; 0 =
                             default (~2^22 polls with back-off, about a
                             second); a wait that runs out sets
                             VL_ERR_TIMEOUT in the result's status word;
                             negative = every wait expires at once (to
                             exercise the timeout path) */
  int64_t memory_budget;  /* bytes the server may hold; 0 = free HBM minus
                             a reserve */
  int32_t tile_rows;      /* 0 = autotune; else rows per fused tile */
  int32_t tile_words;     /* 0 = autotune; else 32-px words per fused tile */
  int32_t reserved[6];
} vl_config;

/* Fill *cfg with defaults. */
VL_API void vl_config_default(vl_config* cfg);

/* Create a context on cfg->device (cfg may be NULL for defaults).  The
 * context owns a device-memory pool and the formula/plan caches.  Not
 * thread-safe: one host thread per context, except for vl_server_* which
 * run their own thread. */
VL_API vl_status vl_context_create(const vl_config* cfg, vl_context** out);

/* Message of the last error on this context (never NULL; "" if none). */
VL_API const char* vl_last_error(vl_context* ctx);

/* Release any handle returned by this library (context last).  NULL ok. */
VL_API void vl_free(void* handle);

/* ------------------------------------------------------------------ images */

/* A float32 image of `channels` planar channels, H x W each: the model of
 * Sec. 2 with its features (intensity, colour components).  `data` holds
 * channels*h*w floats, channel-major then row-major, on the host
 * (data_on_device = 0) or the device (1).  The library copies it into its
 * own padded device layout on `stream` (the copy is ordered on the stream;
 * the caller may reuse host memory once the stream reaches it).
 * Errors: VL_ERR_ARG for h, w, channels < 1 or > 65535, NULL data. */
VL_API vl_status vl_image_create(vl_context* ctx, int32_t h, int32_t w,
                                 int32_t channels, const float* data,
                                 int32_t data_on_device, void* stream,
                                 vl_image** out);

/* Pixel formats of number images. */
typedef enum { VL_PX_F32 = 0, VL_PX_U16 = 1 } vl_pixel_format;

/* The same for 16-bit unsigned pixels (the tool's native precision, Sec.
 * 3): `data` holds channels*h*w uint16 values, kept as uint16 on the device
 * (2 bytes per pixel); a pixel is its integer value, which thresholds,
 * percentiles and number terms read exactly as a float32.  Errors as
 * vl_image_create. */
VL_API vl_status vl_image_create_u16(vl_context* ctx, int32_t h, int32_t w,
                                     int32_t channels, const uint16_t* data,
                                     int32_t data_on_device, void* stream,
                                     vl_image** out);

/* A binary image used directly as an atomic proposition (the paper's atoms
 * "correspond to binary images", Sec. 2).  `data` is h*w bytes (nonzero =
 * true), host or device. */
VL_API vl_status vl_mask_create(vl_context* ctx, int32_t h, int32_t w,
                                const uint8_t* data, int32_t data_on_device,
                                void* stream, vl_image** out);

/* Same, from an already bit-packed mask (h * Wp uint32 words, layout as at
 * the top of this file; padding bits are cleared by the library). */
VL_API vl_status vl_mask_create_packed(vl_context* ctx, int32_t h, int32_t w,
                                       const uint32_t* words,
                                       int32_t data_on_device, void* stream,
                                       vl_image** out);

/* Shape of an image: any output pointer may be NULL.  is_mask = 1 for
 * images made by vl_mask_create*. */
VL_API vl_status vl_image_info(const vl_image* img, int32_t* h, int32_t* w,
                               int32_t* channels, int32_t* is_mask);

/* Pixel format (vl_pixel_format) of a number image; VL_ERR_ARG for masks. */
VL_API vl_status vl_image_format(const vl_image* img, int32_t* format);

/* ----------------------------------------------------------------- volumes
 * The logic of Sec. 2 on D x H x W voxel grids (the paper's 3D outlook,
 * Sec. 1 and Sec. 5).  A volume is stored as its D slices stacked into one
 * image of D*h rows (slice z = rows z*h .. z*h + h - 1); vl_image_info
 * reports h as D*h and vl_image_depth gives D.  Formulas over volumes are
 * compiled with adjacency 26 (the 3 x 3 x 3 cube: voxels differing by at
 * most 1 in every coordinate) or 6 (the faces: differing by 1 in exactly
 * one coordinate); N, rho and labelling then use it, clipped at the
 * volume's border.  Volumes evaluate in the per-operator form (vl_eval
 * takes it whatever the context's exec_mode; vl_eval_batch and the server
 * refuse them).  Results hold D*h x Wp words per root (slice after slice);
 * vl_result_depth gives D.  A percentile ranks all D*h*w values of the
 * channel.  vl_ccl with connectivity 6 or 26 labels a mask volume: label =
 * the minimum linear index z*h*w + y*w + x of the component, -1 for
 * background.
 *   data: channels*d*h*w values (channel-major, then slice, row, column),
 *   host or device as for vl_image_create.
 * Errors: VL_ERR_ARG for sizes < 1, d*h > 2^20, w > 65535 or more than
 * 2^31 - 1 voxels. */
VL_API vl_status vl_volume_create(vl_context* ctx, int32_t d, int32_t h, int32_t w,
                                  int32_t channels, const float* data,
                                  int32_t data_on_device, void* stream,
                                  vl_image** out);
VL_API vl_status vl_volume_create_u16(vl_context* ctx, int32_t d, int32_t h, int32_t w,
                                      int32_t channels, const uint16_t* data,
                                      int32_t data_on_device, void* stream,
                                      vl_image** out);
/* A binary volume (d*h*w bytes, nonzero = true) used as an atom. */
VL_API vl_status vl_mask_volume_create(vl_context* ctx, int32_t d, int32_t h, int32_t w,
                                       const uint8_t* data, int32_t data_on_device,
                                       void* stream, vl_image** out);
/* Depth D of an image (1 for a 2D image) or of a result. */
VL_API vl_status vl_image_depth(const vl_image* img, int32_t* d);
VL_API vl_status vl_result_depth(const vl_result* res, int32_t* d);

/* ---------------------------------------------------------------- formulas */

/* Operators of a formula node.  The primitive ones follow Eq. (1) of Sec. 2;
 * the derived ones are expanded by the compiler into primitives:
 *   OR(a,b)         = not(not a and not b)
 *   INTERIOR(a)     = not N not a                    (erosion, Sec. 2)
 *   SURROUNDED(a,b) = a and not rho(not(a or b))[not b]
 *   GROW(a,b)       = a or (b and rho a[b])           (Sec. 4.2)
 *   TOUCH(a,b)      = a and rho b[a]
 * Atoms: THR_GT / THR_LT compare channel `channel` of image `image` with the
 * float32 constant `t`, strictly; PCT_GT / PCT_LT compare it with that
 * channel's percentile: the value of rank floor(q*(n-1)) in ascending order
 * of its n = H*W values (the "percentiles" normalisation of Sec. 4.2); MASK
 * reads the binary image `image`; TRUE / FALSE are constants. */
typedef enum {
  VL_OP_TRUE = 0, VL_OP_FALSE = 1, VL_OP_THR_GT = 2, VL_OP_THR_LT = 3,
  VL_OP_PCT_GT = 4, VL_OP_PCT_LT = 5, VL_OP_MASK = 6, VL_OP_NOT = 7,
  VL_OP_AND = 8, VL_OP_NEAR = 9, VL_OP_REACH = 10, VL_OP_OR = 11,
  VL_OP_INTERIOR = 12, VL_OP_SURROUNDED = 13, VL_OP_GROW = 14,
  VL_OP_TOUCH = 15,
  /* number terms (the tool's basic arithmetic, Sec. 3) */
  VL_OP_VALUE = 16, VL_OP_ADD = 17, VL_OP_SUB = 18, VL_OP_MUL = 19,
  VL_OP_DIV = 20
} vl_op;

/* Number terms.  Besides masks, a formula may compute number images pixel by
 * pixel and compare them:
 *   VALUE             = channel `channel` of image `image`, as numbers (a
 *                       uint16 pixel is its integer value);
 *   ADD/SUB/MUL/DIV   = a (+ - * /) b for two number terms a, b, or
 *                       a (op) t for the float32 constant t when b = -1;
 * each an IEEE-754 binary32 operation rounded to nearest even, once per
 * node (never fused with another node's operation).  A THR_* or PCT_* node
 * with a >= 0 compares the number term a (instead of image / channel): NaN
 * satisfies no threshold and sorts after +infinity in a percentile.  Number
 * terms are operands of arithmetic and comparisons only; connectives and
 * roots take masks (VL_ERR_FORMULA otherwise).  A plan evaluates all the
 * number terms its comparisons need in one pass over the pixels (at most
 * 16 live values and 1024 operations per formula, else VL_ERR_FORMULA). */

/* One node (32 bytes).  Operands a, b index earlier nodes of the same array
 * (a, b < own index; -1 when unused).  For REACH, a = phi1 (the target) and
 * b = phi2 (the intermediate pixels).  Thresholds and percentiles use a only
 * to compare a number term; arithmetic uses b = -1 for a constant t. */
typedef struct {
  int32_t op;
  int32_t a;
  int32_t b;
  int32_t image;    /* index into the image list given at evaluation */
  int32_t channel;  /* channel of that image (threshold atoms) */
  float t;          /* threshold constant (THR_*) */
  double q;         /* percentile level in [0, 1] (PCT_*) */
} vl_node;

/* Compile a formula DAG given as `n_nodes` nodes in topological order and
 * `n_roots` output node indices (a root may be any node; Sec. 3.2 "output
 * instructions").  connectivity is 4 or 8 for images, 6 or 26 for volumes,
 * and governs both N and the paths of rho.  The compiler expands derived operators, shares identical
 * sub-expressions, and plans fused execution.  Host-only; no device work.
 * Errors: VL_ERR_FORMULA (operand out of order, unknown op, bad arity,
 * percentile level outside [0,1]), VL_ERR_ARG.  ctx may be NULL: the plan is
 * then made for the default tile configuration (a formula is only
 * evaluated by contexts with the tile configuration it was planned for). */
VL_API vl_status vl_formula_compile(vl_context* ctx, const vl_node* nodes,
                                    int32_t n_nodes, const int32_t* roots,
                                    int32_t n_roots, int32_t connectivity,
                                    vl_formula** out);

/* Compile a specification text in the command language of the paper's tool
 * (Sec. 3: commands let / load / save; expressions are numbers, names,
 * applications f(e1, ..., eN), infix applications and parenthesised
 * expressions; macros are expanded, sharing identical sub-expressions).
 * The paper defers the grammar to the tool's documentation; this library
 * reads it as follows.
 *   load x = "s"            x names the next image given at evaluation
 *                           (images in load order; "s" only labels it)
 *   let x = e               a constant
 *   let f(p1, ..., pN) = e  a macro; a body sees its parameters and the
 *                           names defined before it is applied
 *   save "s" e              an output: the mask e (roots in save order)
 *   import "s"              accepted and ignored (derived operators are
 *                           built in)
 *   // ...                  a comment, to the end of the line
 * Expressions, loosest binding first: a | b (or), a & b (and), a >. t and
 * a <. t (strict comparisons of a number term with a number or with
 * percentile(a, q), not chained), + and -, * and /, prefix ! (not) and -.
 * Functions: intensity(x) (channel 0 of image x), red, green, blue, alpha
 * (channels 0-3), channel(x, c), mask(x) (a binary image as an atom),
 * percentile(term, q) (q in [0, 1], only as a comparison's bound), not,
 * and, or, near or N, interior, surrounded(a, b), grow(a, b), touch(a, b),
 * reach or rho(a, b) (= rho a[b]); tt and ff are the constants.  Numbers
 * combine exactly and are rounded to float32 where a node takes them;
 * t - term is computed as (term * -1) + t, and number / term is refused.
 * connectivity as for vl_formula_compile.  err_buf (err_len bytes, may be
 * NULL) receives "" or the error, "line L, column C: ..." for the text.
 * Errors: VL_ERR_FORMULA (syntax, unknown or redefined names, a value of
 * the wrong kind, nothing saved, and the compiler's own checks), VL_ERR_ARG.
 * ctx may be NULL as for vl_formula_compile. */
VL_API vl_status vl_formula_compile_text(vl_context* ctx, const char* src,
                                         int32_t connectivity, vl_formula** out,
                                         char* err_buf, int32_t err_len);

/* Names of a formula compiled from a text: which = 0 its loads (the image
 * order), 1 its saves (the root order), 2 the strings of its loads (what
 * each load names, in image order).  *count (may be NULL) receives how
 * many; with buf non-NULL, name `index` is copied there (NUL-terminated,
 * cut to len - 1 bytes).  A formula compiled from nodes has none.  Errors:
 * VL_ERR_ARG (bad handle, which or index). */
VL_API vl_status vl_formula_spec_names(const vl_formula* f, int32_t which, int32_t* count,
                                       int32_t index, char* buf, int32_t len);

/* Introspection of a compiled plan (debugging and host-side tests).  Call
 * with NULL arrays to get the sizes, then again with arrays of at least
 * those lengths.  Steps run in order; a step of kind 1 (fused group) runs
 * its instructions on every tile; kinds 2, 3 and 5 are the three passes of
 * a batch of component selects (tile labelling, border merge, final
 * select; kind 4 is not used); kind 0 computes percentiles; kind 6 computes rank codes
 * (below); kind 7 evaluates number terms (vl_formula_arith).  Steps are
 * listed in an order that respects their dependencies
 * (vl_formula_step_deps).  Instruction opcodes: 1 threshold, 2 load slot, 3 not, 4 and,
 * 5 or, 6 N, 7 constant, 8 store slot, 9 and-not, 10 threshold by rank
 * code; bit 7 (0x80) of the opcode marks an instruction that a block
 * barrier precedes (each buffer word has one owning thread, and the
 * compiler puts a barrier only where a thread would touch a word another
 * thread touched since the last one).  Slots: [0, n_inter) intermediates, then one per distinct root,
 * then one per mask image.
 *
 * Rank codes (an evaluation strategy, not part of the logic): when many
 * constant thresholds read one image channel, the compiler makes a table
 * of their distinct values t_1 < ... < t_m, and a pixel value v gets the
 * code c = 2 * #{k : t_k < v} + [v equals some t_k] (0 for NaN).  Then
 * v > t_k exactly when c >= 2k, and v < t_k exactly when v is not NaN and
 * c < 2k - 1; an opcode-10 instruction holds the table (a), the bound
 * (image, read as uint16), the code bits (channel), the table's first
 * plane (slot) and the direction (b).
 * The results are those of the strict float comparisons (Sec. 2 atoms). */
typedef struct {
  int32_t n_steps, n_insns, n_selects, n_pct;
  int32_t n_inter_slots, n_root_slots, n_mask_slots, n_roots;
  int32_t n_rank_tables, n_rank_values, n_rank_planes, n_deps;
} vl_plan_sizes;
typedef struct {
  int32_t kind, insn_off, insn_cnt, halo, sel_off, sel_cnt, pct_off, pct_cnt;
  int32_t rank_mask;  /* groups: rank tables their opcode-10 instructions read */
  int32_t rank_halo;  /* groups: largest halo of those instructions */
  int32_t n_bufs;     /* groups: tile buffers the instructions use (0 .. n_bufs-1) */
} vl_plan_step;
typedef struct {
  uint8_t op, dst, a, b;   /* b: direction (1 = less-than) for thresholds, value for constants */
  int16_t halo, slot, image, channel;
  float t;
} vl_plan_insn;
typedef struct {
  int16_t phi1_slot, phi2_slot, z_slot, scratch;
} vl_plan_select;
typedef struct {
  int16_t image, channel, slot, pad;
  double q;
} vl_plan_pct;

VL_API vl_status vl_formula_plan(const vl_formula* f, vl_plan_sizes* sizes,
                                 vl_plan_step* steps, vl_plan_insn* insns,
                                 vl_plan_select* selects, vl_plan_pct* pct,
                                 int32_t* root_slots, int32_t* mask_slot_images);

/* Step dependencies of a plan: step s may start once every step in
 * deps[dep_off[s] .. dep_off[s + 1]) has finished (dep_off has n_steps + 1
 * entries, deps n_deps).  They cover reads after writes, and writes after
 * the reads and the write of a slot's previous value (slots are reused), so
 * any order that respects them computes the same masks; the persistent
 * executor lets independent steps overlap.  Either array may be NULL. */
VL_API vl_status vl_formula_step_deps(const vl_formula* f, int32_t* dep_off, int32_t* deps);

/* Rank tables of a plan (n_rank_tables entries) and their sorted threshold
 * values (n_rank_values floats; table k owns values [value_off, value_off +
 * m)); planes [plane0, plane0 + nbits) hold code bits 0.., plane0 + nbits
 * the NaN pixels.  Either array may be NULL. */
typedef struct {
  int32_t image, channel, m, nbits, value_off, plane0;
} vl_plan_rank;
VL_API vl_status vl_formula_rank_tables(const vl_formula* f, vl_plan_rank* tables,
                                        float* values);

/* Number terms of a plan: one straight-line program run on every pixel
 * (step kind 7, first in the plan).  Opcodes: 0 load channel `channel` of
 * image `image` into register dst; 1-4 dst = a (+ - * /) b, b = 255 for
 * the constant c; 5 store register a into number image `image` (counted
 * from the first one).  Number images follow the formula's own images in
 * a job's image list: thresholds, percentiles and rank tables of a plan
 * name them with index *first_number_image + k.  Any pointer may be NULL;
 * insns receives *n_insns entries. */
typedef struct {
  uint8_t op, dst, a, b;
  int16_t image, channel;
  float c;
} vl_plan_arith;
VL_API vl_status vl_formula_arith(const vl_formula* f, vl_plan_arith* insns, int32_t* n_insns,
                                  int32_t* n_number_images, int32_t* first_number_image);

/* Counts of a compiled formula (any pointer may be NULL):
 *   n_primitive -- primitive nodes (threshold, not, and, N, rho, constants,
 *                  masks) after derived-operator expansion and sharing,
 *                  before any algebraic simplification: the unit of the
 *                  pixel-operation throughput metric;
 *   n_reach     -- rho nodes among them;
 *   n_roots     -- outputs;
 *   n_images    -- 1 + the largest image index the formula reads. */
VL_API vl_status vl_formula_info(const vl_formula* f, int64_t* n_primitive,
                                 int64_t* n_reach, int32_t* n_roots,
                                 int32_t* n_images);

/* Plan statistics (for accounting and benchmarks). */
typedef struct {
  int64_t n_primitive;      /* as vl_formula_info */
  int64_t n_reach;
  int64_t n_threshold;      /* threshold / percentile atoms */
  int64_t n_not, n_and, n_near;
  int32_t n_roots;
  int32_t n_images;
  int32_t n_steps;          /* executor steps (groups + 4 per select batch + percentiles) */
  int32_t n_groups;         /* fused tile groups */
  int32_t n_selects;        /* component selects (one per rho after sharing) */
  int32_t n_channels_read;  /* distinct (image, channel) pairs read by thresholds */
  int64_t mask_writes;      /* masks written to global memory per evaluation */
  int64_t mask_reads;       /* masks read back from global memory per evaluation */
  int32_t max_halo;         /* largest halo of a fused group */
  int32_t n_number_images;  /* number images the arithmetic step writes */
} vl_formula_stats;

VL_API vl_status vl_formula_stats_get(const vl_formula* f, vl_formula_stats* st);

/* -------------------------------------------------------------- evaluation */

/* Evaluate `f` on the images imgs[0..n_imgs) (all H x W; node.image indexes
 * this list; threshold atoms need float images, MASK atoms mask images).
 * Enqueues all work on `stream` and returns without waiting; *out receives
 * a result handle that owns one device mask per root.  The execution form is
 * the context's exec_mode.  Errors: VL_ERR_SHAPE, VL_ERR_ARG, VL_ERR_OOM,
 * VL_ERR_CUDA; device-side errors surface at vl_result_sync. */
VL_API vl_status vl_eval(vl_context* ctx, const vl_formula* f,
                         vl_image* const* imgs, int32_t n_imgs, void* stream,
                         vl_result** out);

/* Same with an explicit execution form (vl_exec_mode). */
VL_API vl_status vl_eval_mode(vl_context* ctx, const vl_formula* f,
                              vl_image* const* imgs, int32_t n_imgs,
                              int32_t exec_mode, void* stream,
                              vl_result** out);

/* One (formula, images) pair of a batch. */
typedef struct {
  const vl_formula* formula;
  vl_image* const* images;
  int32_t n_images;
  int32_t reserved;
} vl_job;

/* Evaluate many jobs (images of different sizes allowed between jobs) in
 * one persistent launch; outs[i] receives job i's result.  When the
 * context's use_graphs is set, the launch sequence is captured into a CUDA
 * graph cached by the batch's structure and replayed.  A batch of a single
 * job may run its per-operator kernels instead, captured the same way, when
 * the tile table (vl_autotune) measured that faster or the formula has at
 * most 24 primitives (after expansion and sharing): a handful of kernels
 * beats a chain of executor steps (vl_eval_mode with VL_EXEC_FUSED always
 * takes the persistent launch).  Enqueue only. */
VL_API vl_status vl_eval_batch(vl_context* ctx, const vl_job* jobs,
                               int32_t n_jobs, void* stream, vl_result** outs);

/* Prepared batches: the jobs' plans, device tables, scratch and result
 * buffers are set up once; vl_batch_run replays the whole batch (one
 * persistent launch, through a cached CUDA graph when the context's
 * use_graphs is set) on the same images and into the same result buffers.
 * The images must stay alive as long as the batch.  Results are borrowed:
 * valid until vl_free(batch), never freed by the caller. */
typedef struct vl_batch vl_batch;
VL_API vl_status vl_batch_prepare(vl_context* ctx, const vl_job* jobs, int32_t n_jobs,
                                  void* stream, vl_batch** out);
VL_API vl_status vl_batch_run(vl_batch* b, void* stream);
VL_API vl_status vl_batch_result(vl_batch* b, int32_t job, vl_result** out);

/* Step timeline of the last run of a batch made by a context with `trace`
 * set: for every (job, step) seven int64 values {job, step, kind, start_ns,
 * end_ns, busy_ns, wait_ns} -- kind as in vl_plan_step, start/end from the
 * device global timer, busy = summed time of its work items, wait = summed
 * time its items spent waiting for the previous step.  Waits for the batch's
 * work.  Writes up to max_entries entries; *n_entries gets the total. */
VL_API vl_status vl_batch_trace(const vl_batch* b, int64_t* out, int64_t max_entries,
                                int64_t* n_entries);

/* Shape of a batch launch: work items, CTAs, dynamic shared memory. */
VL_API vl_status vl_batch_info(const vl_batch* b, int64_t* n_items, int32_t* grid,
                               int64_t* smem_bytes);

/* ---- Tile autotuning.  The paper runs one kernel per operator over whole
 * images (Sec. 3.2) and has no tiles to tune; here the fused groups of a
 * batch run on tiles of rows x 32-px words, and how many tiles a step has
 * decides how well one launch fills the GPU (few large images want small
 * tiles, thousands of small ones large tiles).  With tile_rows = tile_words
 * = 0 in vl_config, every batch takes the shape this table gives for its
 * signature (the set of formulas, and the number, total and largest sizes
 * of its images, in powers of two), else a heuristic (for a batch of one
 * job with at most 24 primitives the per-operator form, else the largest
 * shape whose tiles per step reach three quarters of the persistent grid).
 * A choice of 0 x 0 tiles with 0 CTAs per SM stands for the per-operator
 * form: the batch's single job runs one kernel per primitive, captured in
 * the batch's graph (the autotuner tries it for batches of one job). */
typedef struct {
  int32_t tile_rows;    /* rows per fused-group tile */
  int32_t tile_words;   /* 32-px words per fused-group tile */
  int32_t ctas_per_sm;  /* persistent CTAs per SM */
  int32_t status;       /* VL_OK, or the status that ruled this shape out */
  double ms;            /* mean time of one batched launch (-1: not timed) */
} vl_tile_choice;

/* Time `jobs` under every candidate tile shape and CTAs-per-SM count that
 * fits -- the fixed shapes 32x32, 64x16, 32x16, 16x32, 16x16, 64x8, 32x8,
 * 16x8 (rows x words) and, for a batch of one job, per tile width of 32 and
 * 16 words the lowest height whose tiles fit one wave of the grid (2048 x
 * 2048 on 152 SMs: 14x32 and 27x16) -- and for a batch of one job its
 * per-operator form (reps timed
 * launches each, every one after a 192 MB write that clears the L2, after
 * untimed launches whose device status must be VL_OK; the library holds
 * that scratch while tuning), keep the fastest in the context's table for the
 * batch's signature and return it in *best.  trials (host, max_trials
 * entries, may be NULL) receives every candidate; *n_trials their count.
 * Runs on `stream` and synchronises it; the jobs' results are computed and
 * discarded.  VL_ERR_ARG if the context has a fixed tile shape. */
VL_API vl_status vl_autotune(vl_context* ctx, const vl_job* jobs, int32_t n_jobs, void* stream,
                             int32_t reps, vl_tile_choice* trials, int32_t max_trials,
                             int32_t* n_trials, vl_tile_choice* best);

/* The shape vl_batch_prepare would use for `jobs` now; *tuned = 1 when it
 * comes from a measurement (vl_autotune or vl_tune_load), 0 otherwise. */
VL_API vl_status vl_tile_shape(vl_context* ctx, const vl_job* jobs, int32_t n_jobs,
                               vl_tile_choice* out, int32_t* tuned);

/* Write / merge the context's table of measured shapes to / from a text
 * file (one "signature rows words ctas_per_sm ms" line per entry).  Entries
 * are specific to the GPU model they were measured on; load refuses a file
 * whose header names another SM count (VL_ERR_ARG). */
VL_API vl_status vl_tune_save(vl_context* ctx, const char* path);
VL_API vl_status vl_tune_load(vl_context* ctx, const char* path);

/* Wait for the result's work and return its device status word: VL_OK,
 * VL_ERR_TIMEOUT (a bounded device wait ran out) or VL_ERR_INTERNAL. */
VL_API vl_status vl_result_sync(vl_result* res);

/* Wait, then the raw device status word: 0, VL_ERR_TIMEOUT, or VL_ERR_INTERNAL
 * in the low byte with the failed check in bits 8.. (1 global find bound,
 * 2 global union bound, 3 not used, 4 saved tile state out of range, 5 tile
 * strip-run capacity, 6 shared union-find bound, 7 global union-find entry
 * outside its array). */
VL_API vl_status vl_result_status_word(vl_result* res, int32_t* word);

/* Shape of a result (any pointer may be NULL); words_per_row = Wp. */
VL_API vl_status vl_result_info(const vl_result* res, int32_t* h, int32_t* w,
                                int32_t* words_per_row, int32_t* n_roots);

/* Copy root `root`'s mask (h * Wp uint32 words) to dst, host or device,
 * ordered on `stream` (host copies complete before returning). */
VL_API vl_status vl_result_mask(const vl_result* res, int32_t root,
                                uint32_t* dst, int32_t dst_on_device,
                                void* stream);

/* All roots at once: root r goes to dst + r * h * Wp words (host or
 * device); one host wait at the end for host destinations. */
VL_API vl_status vl_result_masks(const vl_result* res, uint32_t* dst,
                                 int32_t dst_on_device, void* stream);

/* Same, unpacked to h * w bytes of 0/1 by a device kernel. */
VL_API vl_status vl_result_mask_u8(const vl_result* res, int32_t root,
                                   uint8_t* dst, int32_t dst_on_device,
                                   void* stream);

/* Device pointer of root `root`'s packed mask (valid until the result is
 * freed). */
VL_API vl_status vl_result_device_ptr(const vl_result* res, int32_t root,
                                      const uint32_t** ptr);

/* ------------------------------------------------- connected components */

/* Full connected component labelling of a mask image (the operation rho
 * reduces to, Sec. 3.2-3.3): labels_dev receives H*W int32 labels (minimum
 * linear index per component, -1 background).  labels_dev is a caller-owned
 * device buffer of at least H*W int32.  Union-find: tile-local labelling in
 * shared memory, then a global merge with atomics.  A mask volume takes
 * connectivity 6 or 26 (labels = minimum linear index of the 3D component;
 * see the volumes section).  Enqueue only; device errors are reported by
 * vl_ccl_status. */
VL_API vl_status vl_ccl(vl_context* ctx, const vl_image* mask,
                        int32_t connectivity, int32_t* labels_dev,
                        void* stream);

/* The paper's own labelling (Sec. 3.3, Alg. 1), for comparison: labels are
 * pixel indices; every set pixel starts with its own; a main iteration
 * gives pixel p the largest label around the pixel its label names
 * (pointer jumping); every `period` main iterations (0: 16, the period the
 * paper's text gives) a reconnect step raises, by atomic maximum, the label
 * of the pixel that p's label names to the largest label around p; then a
 * termination check (no set pixel has a set neighbour with another label)
 * is read back by the host.  On return labels_dev (device, h*w int32) holds,
 * for every set pixel, the index of one pixel of its component (the same
 * for the whole component), -1 for background: the same partition as
 * vl_ccl, under other label values.  Synchronous: waits for `stream` once
 * per round.  *iterations (may be NULL) receives the number of main
 * iterations.  VL_ERR_TIMEOUT if max_rounds rounds (0: 65536) did not
 * converge; VL_ERR_ARG for a non-mask image, a null buffer or connectivity
 * other than 4 or 8. */
VL_API vl_status vl_ccl_pointer_jumping(vl_context* ctx, const vl_image* mask,
                                        int32_t connectivity, int32_t period,
                                        int32_t max_rounds, int32_t* labels_dev,
                                        void* stream, int32_t* iterations);

/* Synchronise `stream` and return the status word of the last vl_ccl call
 * on this context (VL_OK, VL_ERR_TIMEOUT, VL_ERR_INTERNAL). */
VL_API vl_status vl_ccl_status(vl_context* ctx, void* stream);

/* The same labelling for callers that cannot allocate device memory (the
 * paper has no counterpart: this is an interface for library users).
 * cudaMalloc synchronises the whole device, some applications reserve all
 * device memory up front, and memory owned by another allocator must not
 * grow behind its back; such callers pass their own buffers and this call
 * allocates nothing, needs no context, and calls no allocating routine.
 *   mask_dev   -- device, h * Wp packed words (layout at the top of this
 *                 file); padding bits (columns >= w) are ignored
 *   labels_dev -- device, h * w int32, written (minimum linear index per
 *                 component, -1 background)
 *   wait       -- 0: enqueue on `stream` and return VL_OK; a device
 *                 status of the call (VL_ERR_TIMEOUT, VL_ERR_INTERNAL) is
 *                 then not reported, since the next call clears it;
 *                 nonzero: wait for the stream and return that status
 * Working memory is one fixed array inside the library (about 5 MiB, held
 * by every GPU that loads the library until exit), shared by all calls on a
 * device: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.  The
 * array keeps the last call's contents; the call clears what must start at
 * zero.  The array's device address is looked up on every call (no cache
 * outlives a device reset).  The first call on a device loads the library's
 * device code and sets a kernel attribute: make it before any stream
 * capture.
 * Limit: ceil(h/32) * ceil(Wp/32) tiles of 16 * min(32, Wp) * 32 entries
 * must fit in 2^20 entries -- any image up to 2048 x 1024 or 1024 x 2048,
 * for example.  Larger images return VL_ERR_SHAPE; bad pointers or sizes
 * VL_ERR_ARG. */
VL_API vl_status vl_ccl_noalloc(const uint32_t* mask_dev, int32_t h, int32_t w,
                                int32_t connectivity, int32_t* labels_dev,
                                int32_t wait, void* stream);

/* ----------------------------------------------------------------- serving */

typedef struct {
  int32_t max_inflight_batches;  /* launches in flight at once (default 2) */
  int32_t max_batch_jobs;        /* jobs per launch (default 256) */
  int64_t memory_budget;         /* bytes; 0 = free HBM minus reserve */
  int64_t batch_window_us;       /* how long to gather arrivals (default 200) */
  int32_t reserved[8];
} vl_server_config;

typedef struct {
  int64_t submitted, completed, cancelled, failed;
  int64_t batches;               /* launches issued */
  int64_t bytes_in_use;          /* device bytes held by admitted queries */
  int64_t peak_bytes;
  double p50_ms, p99_ms;         /* submit -> done latency of completed */
} vl_server_stats;

/* Start a serving loop on its own host thread.  Queries are admitted while
 * their device memory fits the budget and a batch slot is free; admitted
 * queries are packed into persistent launches on rotating streams, so new
 * arrivals run while earlier batches are still on the GPU.  The budget
 * (memory_budget, else the free device memory at creation, after the
 * stream-ordered pool has handed back what it held free, minus a reserve)
 * covers the work in flight; a finished query's result keeps its root
 * masks on the device until the caller frees it, so a client should take
 * and free results as they complete. */
VL_API vl_status vl_server_create(vl_context* ctx, const vl_server_config* cfg,
                                  vl_server** out);

/* Queue a query; returns at once with a ticket.  The images must stay alive
 * until the query completes. */
VL_API vl_status vl_server_submit(vl_server* srv, const vl_formula* f,
                                  vl_image* const* imgs, int32_t n_imgs,
                                  int64_t* ticket);

/* Wait up to timeout_us (-1 = forever) for a ticket.  On VL_OK *out gets
 * the query's result (caller frees it); VL_ERR_BUSY if still running;
 * VL_ERR_CANCELLED if cancelled; other codes for failed queries. */
VL_API vl_status vl_server_wait(vl_server* srv, int64_t ticket,
                                int64_t timeout_us, vl_result** out);

/* Cancel a queued query (no effect once it has been launched). */
VL_API vl_status vl_server_cancel(vl_server* srv, int64_t ticket);

VL_API vl_status vl_server_stats_get(vl_server* srv, vl_server_stats* st);

#ifdef __cplusplus
}
#endif
#endif /* VL_H_ */
