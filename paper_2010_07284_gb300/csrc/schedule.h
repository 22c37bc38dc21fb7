// Order of the persistent executor's work list (host only).
//
// The executor's CTAs pop work items in list order, and an item waits for
// every step its own step depends on; so any order in which everything an
// item waits for comes earlier is free of deadlock, whatever the number of
// CTAs.  Which such order runs fastest is what this file decides.
#pragma once
#include <stdint.h>

#include <vector>

#include "vl_internal.h"

namespace vl {

// One step of a job: its items (n of them, consecutive in the pending list
// from `first`), and the estimated time of one item in microseconds.
struct SchedStep {
  int first, n;
  double item_us;
};

// One job: its steps in plan order, and their dependencies as the plan
// lists them (steps dep_off[s] .. dep_off[s + 1] - 1 of `deps`, job-relative
// indexes of earlier steps).
struct SchedJob {
  std::vector<SchedStep> steps;
  const int32_t* dep_off;
  const int32_t* deps;
};

// Put `pending` (every item, job by job and step by step) in executor order
// on a grid of `grid` CTAs:
//   one job   -- a list-scheduling simulation: a CTA that frees up takes the
//                ready item whose step has the longest estimated path to the
//                end of the job (its bottom level); items are emitted in the
//                order the simulation starts them;
//   several   -- by the start time of each step had its job run alone with
//                unlimited CTAs, so that jobs of different sizes interleave by
//                their progress and small jobs finish early.
// Returns false (out untouched) if some item could not be placed, which
// dependency lists that only point at earlier steps rule out.
bool order_work_items(const std::vector<SchedJob>& jobs, const std::vector<WorkItem>& pending,
                      int grid, std::vector<WorkItem>* out);

}  // namespace vl
