// ops.h -- per-size kernel tables (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "kkt_scan.cuh"
#include "residual.cuh"
#include "sqp.cuh"
#include "scan_rows.cuh"
#include "riccati_cta.cuh"

namespace pdl {

static constexpr size_t kSmemMax = kSmemCta;  // opt-in shared memory per CTA (sm_103a)

struct SizeOps {
    int n, m;
    cudaError_t (*scan)(const KktArgs&, int warps, cudaStream_t);
    cudaError_t (*riccati)(const KktArgs&, cudaStream_t);
    cudaError_t (*resid)(const ResidArgs&, cudaStream_t);
    size_t (*scan_smem)(int warps);
    // SRBD model (n = m = 12 nrob); null for other sizes
    cudaError_t (*linearize)(const LinArgs&, cudaStream_t);
    cudaError_t (*merit)(const MeritArgs&, cudaStream_t);
    cudaError_t (*sqp)(const SqpArgs&, int warps, cudaStream_t);
    size_t (*sqp_smem)(int warps);
    cudaError_t (*scan_checked)(const KktArgs&, int warps, int64_t limit, cudaStream_t);
    int lq_stage_floats;   // floats of one linearised stage kept by the fused SQP
    // floats of global workspace per CTA when the scan's work areas do not fit
    // in shared memory (0: they fit)
    size_t (*scan_gws_floats)(int warps);
    int unit_warps;        // warps per horizon chunk; warps x unit_warps <= 32
    size_t lin_ws_floats;  // global workspace of the standalone linearisation (0: none)
    // the split scan (one CTA per horizon chunk, W = 8 or 16; sizes whose
    // chunks are 8-warp units) and its global workspace per instance; null /
    // 0 for other sizes
    cudaError_t (*scan_split)(const KktArgs&, int warps, cudaStream_t);
    size_t (*scan_split_gws_floats)(int warps);
    // merit, filter decision and update of the unfused SQP iteration that
    // split plans run (SRBD sizes); null for other sizes
    cudaError_t (*sqp_step)(const SqpStepArgs&, cudaStream_t);
};

// Warp counts (horizon chunks) a size supports: 1, 4, 8 or 16 within the
// 1024-thread block limit.
inline bool warps_ok(const SizeOps* o, int w)
{
    return (w == 1 || w == 4 || w == 8 || w == 16) && w * o->unit_warps <= 32;
}

// The kernel table of an (n, m) size, or null when it is not instantiated.
const SizeOps* find_ops(int n, int m);

// Tables of the instantiated sizes (one translation unit each).
const SizeOps* ops_small(int n, int m);   // (1,1) (2,1) (3,2) (4,2)
const SizeOps* ops_12(int n, int m);      // (12,12): SRBD, fused SQP
const SizeOps* ops_24(int n, int m);      // (24,24): two stacked robots
const SizeOps* ops_36(int n, int m);      // (36,24): Riccati comparator, residual
const SizeOps* ops_48(int n, int m);      // (48,48): four robots
const SizeOps* ops_96(int n, int m);      // (96,96): eight robots
const SizeOps* ops_192(int n, int m);     // (192,192): sixteen robots

}  // namespace pdl
