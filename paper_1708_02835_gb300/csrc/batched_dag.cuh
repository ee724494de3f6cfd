// Persistent batched scheduler (batched_dag.cu): plan and launch.
#pragma once
#include <vector>

#include "batched.cuh"

namespace egs {

// Device control block of one persistent run (reset before every run).
struct DagCtl {
    unsigned long long next;      // next task to claim
    unsigned abort;               // set when a wait ran out of time
    unsigned timeouts;            // waits that ran out of time
    unsigned long long limit_ns;  // bound of every dependency wait
    long long withhold;           // task whose completion is never signalled (failure tests), -1 = none
};

constexpr unsigned long long kDagWaitLimitNs = 10000000000ull;  // 10 s

// Task list of the FP64 batch with T[p] tiles per side for problem p, in a
// checked topological order; cnt_off[p] = offset of problem p's counters.
egs_status dag_plan(const std::vector<int> &T, int b, std::vector<int4> &tasks, std::vector<size_t> &cnt_off,
                    size_t &ncounters);
// CTAs of the persistent launch (SMs x resident CTAs per SM), 0 on error.
int dag_grid();
cudaError_t dag_enqueue(const int4 *d_tasks, long long ntasks, const BatchProblem *d_probs, DagCtl *d_ctl, int b,
                        int grid, cudaStream_t s);

}  // namespace egs
