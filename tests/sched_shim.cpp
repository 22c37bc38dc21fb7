// Test shim: the executor's work-list order (paper_2010_07284_gb300/csrc/
// schedule.cpp) behind a plain C entry point, compiled with the host
// compiler by tests/test_schedule.py.  Every step's items are one sub-item
// each.
#include "schedule.h"

extern "C" int sched_order(int n_jobs, const int* n_steps, const int* step_n,
                           const double* step_us, const int* dep_off, const int* deps, int grid,
                           int* out_job, int* out_step, int* out_first) {
  std::vector<vl::SchedJob> jobs(n_jobs);
  std::vector<vl::WorkItem> pending;
  int s0 = 0, o0 = 0, d0 = 0;
  for (int j = 0; j < n_jobs; ++j) {
    jobs[j].dep_off = dep_off + o0;
    jobs[j].deps = deps + d0;
    for (int s = 0; s < n_steps[j]; ++s) {
      vl::SchedStep st{(int)pending.size(), step_n[s0 + s], step_us[s0 + s]};
      for (int k = 0; k < st.n; ++k) pending.push_back(vl::WorkItem{j, s, k, 1});
      jobs[j].steps.push_back(st);
    }
    d0 += dep_off[o0 + n_steps[j]];
    o0 += n_steps[j] + 1;
    s0 += n_steps[j];
  }
  std::vector<vl::WorkItem> items;
  if (!vl::order_work_items(jobs, pending, grid, &items)) return -1;
  for (size_t i = 0; i < items.size(); ++i) {
    out_job[i] = items[i].job;
    out_step[i] = items[i].step;
    out_first[i] = items[i].first;
  }
  return (int)items.size();
}
