// Order of the persistent executor's work list (see schedule.h).
#include "schedule.h"

#include <algorithm>
#include <cmath>
#include <queue>

namespace vl {

bool order_work_items(const std::vector<SchedJob>& jobs, const std::vector<WorkItem>& pending,
                      int grid, std::vector<WorkItem>* out) {
  grid = std::max(1, grid);
  // steps of every job in one list
  struct Rec { int job, first, n; double item_us, bl, t0; int deps_left; };
  std::vector<Rec> recs;
  std::vector<int> base(jobs.size() + 1, 0);
  for (size_t j = 0; j < jobs.size(); ++j) {
    base[j] = (int)recs.size();
    const SchedJob& J = jobs[j];
    for (size_t s = 0; s < J.steps.size(); ++s)
      recs.push_back(Rec{(int)j, J.steps[s].first, J.steps[s].n, J.steps[s].item_us, 0.0, 0.0,
                         J.dep_off[s + 1] - J.dep_off[s]});
  }
  base[jobs.size()] = (int)recs.size();
  const auto len = [&](const Rec& r) { return std::ceil((double)r.n / grid) * r.item_us; };
  std::vector<std::vector<int>> succ(recs.size());
  for (size_t j = 0; j < jobs.size(); ++j)
    for (size_t s = 0; s < jobs[j].steps.size(); ++s)
      for (int q = jobs[j].dep_off[s]; q < jobs[j].dep_off[s + 1]; ++q) {
        const int d = jobs[j].deps[q];
        if (d < 0 || d >= (int)s) return false;  // only earlier steps
        succ[base[j] + d].push_back(base[j] + (int)s);
      }
  std::vector<WorkItem> items;
  items.reserve(pending.size());
  if (jobs.size() > 1) {
    // each step's start had its job run alone with unlimited CTAs: the
    // latest estimated finish of its dependencies
    for (size_t j = 0; j < jobs.size(); ++j) {
      std::vector<double> fin(jobs[j].steps.size(), 0.0);
      for (size_t s = 0; s < jobs[j].steps.size(); ++s) {
        double t = 0;
        for (int q = jobs[j].dep_off[s]; q < jobs[j].dep_off[s + 1]; ++q)
          t = std::max(t, fin[jobs[j].deps[q]]);
        Rec& r = recs[base[j] + s];
        r.t0 = t;
        fin[s] = t + len(r);
      }
    }
    std::vector<int> order(recs.size());
    for (size_t r = 0; r < recs.size(); ++r) order[r] = (int)r;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return recs[a].t0 < recs[b].t0; });
    for (int r : order)
      for (int k = 0; k < recs[r].n; ++k) items.push_back(pending[recs[r].first + k]);
  } else {
    // bottom levels: a step's estimated length plus the longest of its
    // successors' (dependencies point at earlier steps: one backward sweep)
    for (int r = (int)recs.size() - 1; r >= 0; --r) {
      double tail = 0;
      for (int x : succ[r]) tail = std::max(tail, recs[x].bl);
      recs[r].bl = len(recs[r]) + tail;
    }
    // the simulation: ready items by bottom level, then list position
    struct Ready {
      double bl; int idx;
      bool operator<(const Ready& o) const { return bl != o.bl ? bl < o.bl : idx > o.idx; }
    };
    struct Busy {
      double t; int rec;
      bool operator<(const Busy& o) const { return t > o.t; }
    };
    std::priority_queue<Ready> ready;
    std::priority_queue<Busy> busy;
    std::vector<int> left(recs.size()), rec_of(pending.size(), -1);
    for (size_t r = 0; r < recs.size(); ++r)
      for (int k = 0; k < recs[r].n; ++k) rec_of[recs[r].first + k] = (int)r;
    auto release = [&](int r) {
      for (int k = 0; k < recs[r].n; ++k) ready.push(Ready{recs[r].bl, recs[r].first + k});
    };
    for (size_t r = 0; r < recs.size(); ++r) {
      left[r] = recs[r].n;
      if (recs[r].deps_left == 0) release((int)r);
    }
    double now = 0;
    int free_ctas = grid;
    while (items.size() < pending.size()) {
      while (free_ctas > 0 && !ready.empty()) {
        const int idx = ready.top().idx;
        ready.pop();
        items.push_back(pending[idx]);
        busy.push(Busy{now + recs[rec_of[idx]].item_us, rec_of[idx]});
        --free_ctas;
      }
      if (busy.empty()) break;  // nothing ready and nothing running
      const Busy b = busy.top();
      busy.pop();
      now = b.t;
      ++free_ctas;
      if (--left[b.rec] == 0)
        for (int x : succ[b.rec])
          if (--recs[x].deps_left == 0) release(x);
    }
  }
  if (items.size() != pending.size()) return false;
  *out = std::move(items);
  return true;
}

}  // namespace vl
