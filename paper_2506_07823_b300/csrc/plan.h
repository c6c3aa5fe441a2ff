// plan.h -- the plan object behind pdilqr_plan (internal to the library).
#pragma once

#include <algorithm>
#include <vector>

#include "ops.h"
#include "pdilqr.h"

struct pdilqr_plan {
    int n = 0, m = 0, count = 0, warps = 0, refine = 0, maxN = 0;
    int ipc = 0;         // instances per CTA of the row-per-lane sequential SQP (0: the solver's own)
    int m64 = 0;         // 1: FP64 elimination of the scan combines' M (n = 36)
    int split = 0;       // 1: the scan's chunks on separate CTAs (kkt_scan_split_kernel)
    unsigned* sbar = nullptr;  // [count] phase counters of the split scan
    // unfused SQP iteration of split plans (SRBD sizes): linearised stages,
    // theta_max, stop flags and dx_0 per instance
    float *lqA = nullptr, *lqB = nullptr, *lqc = nullptr, *lqQ = nullptr, *lqR = nullptr,
          *lqq = nullptr, *lqr = nullptr;
    double* sq_thmax = nullptr;
    int32_t* sq_done = nullptr;
    float* sq_s = nullptr;
    int64_t total = 0;
    const pdl::SizeOps* ops = nullptr;
    std::vector<void*> allocs;
    int32_t* dN = nullptr;
    int64_t* doff = nullptr;
    int32_t* dorder = nullptr;
    int64_t* dstage_inst = nullptr;
    // policy / value function / closed-loop maps per stage
    float *K = nullptr, *k = nullptr, *P = nullptr, *p = nullptr, *Abar = nullptr, *bbar = nullptr;
    // refinement
    float *rq = nullptr, *rr = nullptr, *rc = nullptr, *rs = nullptr;
    float *ddx = nullptr, *ddu = nullptr, *ddl = nullptr, *dk = nullptr, *dp = nullptr;
    double* norms = nullptr;
    int32_t* st2 = nullptr;
    float* lqcache = nullptr;   // linearised stages kept by the fused SQP (SRBD sizes)
    float* gws = nullptr;       // per-CTA scan work areas (sizes beyond shared memory)
    float* lin_ws = nullptr;    // stage areas of the standalone linearisation (large sizes)
    int max_count = 0;   // capacity of the batch tables (capacity plans)
    int dbg = 0;         // test switches (PDILQR_DEBUG_*)
    cudaGraphExec_t graph = nullptr;   // captured solve (pdilqr_solve_capture)

    template <typename T>
    cudaError_t alloc(T** ptr, size_t count_) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, std::max<size_t>(count_, 1) * sizeof(T));
        if (e == cudaSuccess) {
            allocs.push_back(v);
            *ptr = static_cast<T*>(v);
        }
        return e;
    }
    ~pdilqr_plan() {
        if (graph) cudaGraphExecDestroy(graph);
        for (void* v : allocs) cudaFree(v);
    }
};

namespace pdl {

// A plan whose workspace holds `slots` stage slots and whose batch tables hold
// up to `max_count` instances; the batch itself is set per launch.
pdilqr_status plan_create_capacity(int n, int m, int max_count, int64_t slots, int warps,
                                   pdilqr_plan** out);
// Set the batch of a capacity plan from host arrays (pinned for asynchronous
// copies): horizons, first slots and CTA order.  Stream-ordered.
pdilqr_status plan_set_batch_async(pdilqr_plan* pl, const int32_t* hN, const int64_t* hoff,
                                   const int32_t* horder, int count, int maxN, cudaStream_t st);
// Turn a capacity plan created with one warp into a split plan (the scan's
// `warps` horizon chunks of an instance on separate CTAs, an unfused SQP
// iteration): allocates the split scan's work areas and the linearised LQ
// arrays.  Sizes without a split scan or an SRBD step kernel: INVALID_ARG.
pdilqr_status plan_enable_split(pdilqr_plan* pl, int warps);
// Copy the stage-slot -> instance map of the batch (all `slots` entries of
// the capacity, -1 for a slot of no instance) from pinned host memory; the
// split plan's linearisation reads it.  Stream-ordered.
pdilqr_status plan_set_stage_inst_async(pdilqr_plan* pl, const int64_t* hstage, cudaStream_t st);

}  // namespace pdl
