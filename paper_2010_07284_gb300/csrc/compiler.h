// Host compiler: formula node array -> execution plan.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vl.h"
#include "vl_internal.h"

namespace vl {

// Operators of the execution DAG (after expansion and lowering).
enum EOp : int32_t {
  E_TRUE, E_FALSE, E_THR, E_PCT, E_MASK, E_NOT, E_AND, E_OR, E_ANDNOT, E_NEAR,
  E_RZ,   // component select: phi2-components meeting N phi1 (core of rho)
  E_COPY  // identity (a root that is directly an input mask)
};

struct ENode {
  int32_t op;
  int32_t a, b;
  int32_t img, ch;
  int32_t lt;     // threshold direction: 1 for <, 0 for >
  float t;
  double q;
  int32_t pct_slot;
};

struct PlanParams {
  int group_buffers;  // shared-memory tile buffers per group
  int hmax;           // maximum halo (N depth) inside a group
  // a mask slot is reused only by a value defined at least this many steps
  // after the last read of its previous value: reuse adds write-after-read
  // dependencies, which a distant reader keeps off the critical path
  int reuse_distance = 32;
  // select scratch sets (union-find, saved tile state) are handed out round
  // robin from a pool of this many, so consecutive select batches use
  // different sets and need not wait for each other
  int scratch_sets = 64;
};

struct Plan {
  int conn = 8;
  int64_t n_primitive = 0;  // metric unit: primitive nodes after expansion + sharing
  int64_t n_reach = 0;
  int n_roots = 0;
  std::vector<ENode> exec;       // execution DAG, topological
  std::vector<int> exec_roots;   // exec node of each root
  // materialised masks
  int n_inter_slots = 0;         // reusable intermediate slots
  int n_root_slots = 0;          // one per distinct root node
  int n_mask_slots = 0;          // one per mask image index used
  std::vector<int> root_slot;    // slot of each root
  std::vector<int> mask_slot_image;  // image index of each mask slot
  // steps
  std::vector<StepDesc> steps;
  std::vector<Insn> insns;
  std::vector<RzDesc> rz;
  std::vector<PctDesc> pct;
  int n_pct_slots = 0;
  int n_scratch_sets = 0;         // select scratch sets used (allocated per job)
  int max_group_halo = 0;
  // image requirements: kind per image index (0 unused, 1 float, 2 mask)
  std::vector<int> img_kind;
  std::vector<int> img_channels;  // channels needed (max channel + 1)
  PlanParams params{};
  // rank codes (see RankTab): tables, their sorted values, planes per job
  std::vector<RankTab> rtab;
  std::vector<float> rvals;
  int n_planes = 0;
  // step dependencies (CSR): step s may start once every step in
  // deps[dep_off[s] .. dep_off[s+1]) has finished (reads after writes,
  // writes after reads and writes of the same slot, the phases of a select
  // batch, rank codes and percentiles before their readers)
  std::vector<int32_t> dep_off, deps;
  // number terms: one straight-line program over the pixels (SK_ARITH)
  // writes the number images that comparisons read; in a job's image table
  // they follow the formula's own images (index img_kind.size() + k)
  std::vector<ArithInsn> arith;
  int n_num_images = 0;
  int arith_regs = 0;
  // accounting: primitive op counts by kind (threshold, not, and, N, rho,
  // number terms, other)
  int64_t n_thr = 0, n_not = 0, n_and = 0, n_near = 0, n_num = 0, n_other = 0;
};

constexpr int MAX_RZ_BATCH = 32;  // selects of one level run together in one step
// A batch of one job whose plan has at most this many primitives runs the
// per-operator form (captured in the batch's graph) instead of the
// persistent executor: a handful of kernels beats a chain of executor steps.
constexpr int kTinyPlanPrimitives = 24;
// Rank codes: a channel gets a table when at least this many constant
// thresholds read it; tables hold at most kRankMaxValues values (codes fit
// 14 bits) and a formula at most kRankMaxTables tables (one bit each in a
// group's rank_mask).
constexpr int kRankMinThresholds = 4;
constexpr int kRankMaxValues = 8191;
constexpr int kRankMaxTables = 32;

// Returns VL_OK or an error code with a message in *err.
int compile_formula(const vl_node* nodes, int n_nodes, const int32_t* roots, int n_roots,
                    int conn, const PlanParams& pp, Plan* out, std::string* err);

}  // namespace vl
