// ops_impl.cuh -- launch wrappers instantiated per (n, m) in the ops_*.cu units.
// A kernel whose shared memory cannot fit on sm_103a is not instantiated; its
// launcher reports cudaErrorInvalidConfiguration.
#pragma once

#include <atomic>

#include "ops.h"

namespace pdl {

// Dynamic shared memory of a kernel (the carveout stays the driver's choice:
// forcing the largest one takes L1 away from the global-memory reads)
template <class Kern>
static cudaError_t set_smem(Kern kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The shared-memory opt-in is an attribute of the kernel on each device: it
// is set once per (kernel, device) and remembered in a per-kernel bit mask
// of devices.  Setting it is idempotent, so two threads that race on the
// first launch on a device at worst both set it; the bit is published only
// after the call succeeded.
template <class Kern>
static cudaError_t ensure_smem(Kern kernel, size_t bytes, std::atomic<uint64_t>& done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = set_smem(kernel, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}


// W horizon chunks, each owned by UnitWarps<NX> warps; a (W, unit) pair above
// the 1024-thread block limit is not instantiated.
template <int NX, int NU, int W>
static cudaError_t launch_scan_w(const KktArgs& a, cudaStream_t st)
{
    constexpr int UW = UnitWarps<NX>::value;
    using SM = ScanSmem<NX, NU, W>;
    if constexpr (W * UW * 32 > 1024) {
        return cudaErrorInvalidConfiguration;
    } else {
        // work areas in shared memory when they fit, else in the plan's global
        // workspace; the wide units' tile buffers after them when they fit
        constexpr bool GWS = SM::BYTES > kSmemMax;
        constexpr size_t tb = UnitTiles<W, UW>::total(GWS ? 0 : SM::BYTES);
        constexpr size_t bytes = GWS ? UnitFactor<NU, W, UW, NX>::total(tb) : tb;
        if (GWS && !a.gws) return cudaErrorInvalidConfiguration;
        static std::atomic<uint64_t> smem_done{0};
        if (cudaError_t e = ensure_smem(kkt_scan_kernel<NX, NU, W, UW>, bytes, smem_done); e != cudaSuccess)
            return e;
        KktArgs b = a;
        if (!GWS) b.gws = nullptr;
        kkt_scan_kernel<NX, NU, W, UW><<<a.count, W * 32 * UW, bytes, st>>>(b);
        return cudaGetLastError();
    }
}

template <int NX, int NU, int W>
static cudaError_t launch_scan_checked_w(const KktArgs& a, int64_t limit, cudaStream_t st)
{
    using SM = ScanSmem<NX, NU, W>;
    if constexpr (SM::BYTES > kSmemMax) {
        return cudaErrorInvalidConfiguration;
    } else {
    static std::atomic<uint64_t> smem_done{0};
    if (cudaError_t e = ensure_smem(kkt_scan_checked_kernel<NX, NU, W>, SM::BYTES, smem_done); e != cudaSuccess)
        return e;
    kkt_scan_checked_kernel<NX, NU, W><<<a.count, W * 32, SM::BYTES, st>>>(a, limit);
    return cudaGetLastError();
    }
}

template <int NX, int NU>
static cudaError_t launch_scan_checked(const KktArgs& a, int warps, int64_t limit, cudaStream_t st)
{
    switch (warps) {
        case 4: return launch_scan_checked_w<NX, NU, 4>(a, limit, st);
        case 8: return launch_scan_checked_w<NX, NU, 8>(a, limit, st);
        case 16: return launch_scan_checked_w<NX, NU, 16>(a, limit, st);
        default: return cudaErrorInvalidValue;
    }
}

// Floats of global workspace per CTA (0 when the work areas fit in shared
// memory or the warp count is not available for this size).
template <int NX, int NU, int W>
static size_t scan_gws_floats_w()
{
    using SM = ScanSmem<NX, NU, W>;
    if (W * UnitWarps<NX>::value * 32 > 1024) return 0;
    return SM::BYTES > kSmemMax ? SM::TOTAL : 0;
}

template <int NX, int NU>
static size_t scan_gws_floats(int warps)
{
    switch (warps) {
        case 1: return scan_gws_floats_w<NX, NU, 1>();
        case 4: return scan_gws_floats_w<NX, NU, 4>();
        case 8: return scan_gws_floats_w<NX, NU, 8>();
        case 16: return scan_gws_floats_w<NX, NU, 16>();
        default: return 0;
    }
}

template <int NX, int NU>
static size_t scan_smem(int warps)
{
    switch (warps) {
        case 1: return ScanSmem<NX, NU, 1>::BYTES;
        case 4: return ScanSmem<NX, NU, 4>::BYTES;
        case 8: return ScanSmem<NX, NU, 8>::BYTES;
        case 16: return ScanSmem<NX, NU, 16>::BYTES;
        default: return 0;
    }
}

template <int NX, int NU>
static cudaError_t launch_scan(const KktArgs& a, int warps, cudaStream_t st)
{
    switch (warps) {
        case 1: return launch_scan_w<NX, NU, 1>(a, st);
        case 4: return launch_scan_w<NX, NU, 4>(a, st);
        case 8: return launch_scan_w<NX, NU, 8>(a, st);
        case 16: return launch_scan_w<NX, NU, 16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

// Sizes whose sequential recursion runs one 128-thread CTA per instance
// (register-tiled products, column-per-thread elimination); the others run
// one warp per instance.
template <int NX, int NU>
struct UseRicCta {
    static constexpr bool value = NX >= 24 && NX + NU + 1 <= 64 && NX % 6 == 0 && NU % 8 == 0;
};

template <int NX, int NU>
static cudaError_t launch_riccati(const KktArgs& a, cudaStream_t st)
{
    if constexpr (UseRicCta<NX, NU>::value) {
        constexpr size_t bytes = RicCtaL<NX, NU>::BYTES;
        static std::atomic<uint64_t> smem_done{0};
        if (cudaError_t e = ensure_smem(riccati_cta_kernel<NX, NU>, bytes, smem_done); e != cudaSuccess)
            return e;
        riccati_cta_kernel<NX, NU><<<a.count, kRcThreads, bytes, st>>>(a);
        return cudaGetLastError();
    } else {
        using SM = RicSmem<NX, NU>;
        // warps (instances) per block: up to 4, as many as fit in shared memory
        constexpr int FIT = (int)((227 * 1024) / SM::BYTES);
        constexpr int WPB = FIT >= 4 ? 4 : (FIT >= 1 ? FIT : 1);
        constexpr size_t bytes = SM::BYTES * WPB;
        if constexpr (bytes > kSmemMax) {
            return cudaErrorInvalidConfiguration;
        } else {
            static std::atomic<uint64_t> smem_done{0};
            if (cudaError_t e = ensure_smem(riccati_kernel<NX, NU>, bytes, smem_done); e != cudaSuccess)
                return e;
            const int grid = (a.count + WPB - 1) / WPB;
            riccati_kernel<NX, NU><<<grid, 32 * WPB, bytes, st>>>(a);
            return cudaGetLastError();
        }
    }
}

template <int NX, int NU>
static cudaError_t launch_resid(const ResidArgs& a, cudaStream_t st)
{
    if constexpr (ResSmemCfg<NX, NU>::value && NX % 4 == 0 && NU % 4 == 0) {
        using C = ResSmemCfg<NX, NU>;
        static std::atomic<uint64_t> smem_done{0};
        if (cudaError_t e = ensure_smem(kkt_residual_smem_kernel<NX, NU>, C::BYTES, smem_done);
            e != cudaSuccess)
            return e;
        const int64_t blocks = (a.total_stages + C::SPB - 1) / C::SPB;
        kkt_residual_smem_kernel<NX, NU><<<(unsigned)blocks, C::THREADS, C::BYTES, st>>>(a);
        return cudaGetLastError();
    } else {
        const int64_t blocks = (a.total_stages + 7) / 8;
        kkt_residual_kernel<NX, NU><<<(unsigned)blocks, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
}

// Stage slots per block of the standalone linearisation and where its stage
// areas live: four one-warp units in shared memory for small states, one
// unit per block for larger ones, a global workspace beyond shared memory.
template <int NX, int NU>
struct LinCfg {
    static constexpr size_t STAGE_BYTES = sizeof(float) * StageL<NX, NU>::SIZE;
    static constexpr int UW = UnitWarps<NX>::value;
    static constexpr int SPB = (UW == 1 && 4 * STAGE_BYTES <= kSmemMax) ? 4 : 1;
    static constexpr bool GLOBAL = SPB * STAGE_BYTES > kSmemMax;
    static constexpr int GLOBAL_BLOCKS = 2 * 148;   // blocks of the global-workspace form
};

template <int NX, int NU>
static size_t lin_ws_floats()
{
    using C = LinCfg<NX, NU>;
    return C::GLOBAL ? (size_t)C::GLOBAL_BLOCKS * StageL<NX, NU>::SIZE : 0;
}

template <int NX, int NU>
static cudaError_t launch_linearize(const LinArgs& a, cudaStream_t st)
{
    using C = LinCfg<NX, NU>;
    constexpr int THREADS = C::SPB * 32 * C::UW;
    if (a.total <= 0) return cudaSuccess;
    if constexpr (C::GLOBAL) {
        if (!a.work) return cudaErrorInvalidConfiguration;
        const int64_t blocks = std::min<int64_t>(a.total, C::GLOBAL_BLOCKS);
        linearize_kernel<NX, NU, C::SPB, C::UW><<<(unsigned)blocks, THREADS, 0, st>>>(a);
        return cudaGetLastError();
    } else {
        constexpr size_t bytes = C::SPB * C::STAGE_BYTES;
        static std::atomic<uint64_t> smem_done{0};
        if (cudaError_t e = ensure_smem(linearize_kernel<NX, NU, C::SPB, C::UW>, bytes, smem_done); e != cudaSuccess)
            return e;
        LinArgs b = a;
        b.work = nullptr;
        const int64_t blocks = (a.total + C::SPB - 1) / C::SPB;
        linearize_kernel<NX, NU, C::SPB, C::UW><<<(unsigned)blocks, THREADS, bytes, st>>>(b);
        return cudaGetLastError();
    }
}

template <int NX, int NU>
static cudaError_t launch_merit(const MeritArgs& a, cudaStream_t st)
{
    merit_kernel<NX, NU><<<a.count, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <int NX, int NU, int W>
static cudaError_t launch_sqp_w(const SqpArgs& a, cudaStream_t st)
{
    constexpr int UW = UnitWarps<NX>::value;
    using SM = SqpSmem<NX, NU, W>;
    if constexpr (W * UW * 32 > 1024) {
        return cudaErrorInvalidConfiguration;
    } else {
        // scan work areas in shared memory when they fit, else in the plan's
        // global workspace with the line-search extras alone in shared memory
        constexpr bool GWS = SM::SC::BYTES > kSmemMax;
        constexpr size_t tb = UnitTiles<W, UW>::total(GWS ? SM::EXTRA_BYTES : SM::BYTES);
        constexpr size_t bytes = GWS ? UnitFactor<NU, W, UW>::total(tb) : tb;
        if (GWS && !a.ka.gws) return cudaErrorInvalidConfiguration;
        static std::atomic<uint64_t> smem_done{0};
        if (cudaError_t e = ensure_smem(sqp_kernel<NX, NU, W, UW>, bytes, smem_done); e != cudaSuccess)
            return e;
        SqpArgs b = a;
        if (!GWS) b.ka.gws = nullptr;
        sqp_kernel<NX, NU, W, UW><<<a.ka.count, W * 32 * UW, bytes, st>>>(b);
        return cudaGetLastError();
    }
}

// The split scan: W CTAs per instance (one per horizon chunk), launched
// cooperatively after the instances' phase counters are zeroed.  The launch
// is refused (cudaErrorCooperativeLaunchTooLarge) when the W x count CTAs
// cannot all be resident at once, which the phase barriers need.
template <int NX, int NU, int W>
static cudaError_t launch_scan_split_w(const KktArgs& a, cudaStream_t st)
{
    constexpr int UW = UnitWarps<NX>::value;
    if constexpr (UW < 8) {
        return cudaErrorInvalidConfiguration;
    } else {
        constexpr size_t tb = UnitTiles<1, UW>::total(0);
        constexpr size_t bytes = UnitFactor<NU, 1, UW>::total(tb);
        if (!a.gws || !a.sbar || a.count < 1) return cudaErrorInvalidValue;
        auto kern = kkt_scan_split_kernel<NX, NU, W, UW>;
        static std::atomic<uint64_t> smem_done{0};
        if (cudaError_t e = ensure_smem(kern, bytes, smem_done); e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return e;
        if (cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev); e != cudaSuccess)
            return e;
        if (cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * UW, bytes);
            e != cudaSuccess)
            return e;
        if ((int64_t)W * a.count > (int64_t)per_sm * sms) return cudaErrorCooperativeLaunchTooLarge;
        if (cudaError_t e = cudaMemsetAsync(a.sbar, 0, sizeof(unsigned) * a.count, st); e != cudaSuccess)
            return e;
        KktArgs b = a;
        void* args[] = {(void*)&b};
        return cudaLaunchCooperativeKernel((const void*)kern, dim3(W, a.count), dim3(32 * UW), args,
                                           bytes, st);
    }
}

template <int NX, int NU>
static cudaError_t launch_scan_split(const KktArgs& a, int warps, cudaStream_t st)
{
    switch (warps) {
        case 8: return launch_scan_split_w<NX, NU, 8>(a, st);
        case 16: return launch_scan_split_w<NX, NU, 16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int NX, int NU>
static size_t scan_split_gws_floats(int warps)
{
    if (UnitWarps<NX>::value < 8) return 0;
    switch (warps) {
        case 8: return ScanSmem<NX, NU, 8>::TOTAL;
        case 16: return ScanSmem<NX, NU, 16>::TOTAL;
        default: return 0;
    }
}

// The per-instance SQP step (merit, filter, update) of the unfused iteration
template <int NX, int NU>
static cudaError_t launch_sqp_step(const SqpStepArgs& a, cudaStream_t st)
{
    if (a.count < 1) return cudaSuccess;
    sqp_step_kernel<NX, NU><<<a.count, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// The one-chunk (sequential recursion) fused SQP of small SRBD states: the
// row-per-lane kernel, two instances per warp, WPC warps per CTA.
template <int NX, int WPC>
static cudaError_t launch_sqp_rows_w(const SqpArgs& a, cudaStream_t st)
{
    constexpr size_t bytes = WPC * SqpRowsSmem<NX>::BYTES;
    static std::atomic<uint64_t> smem_done{0};
    if (cudaError_t e = ensure_smem(sqp_rows_kernel<NX, WPC>, bytes, smem_done); e != cudaSuccess)
        return e;
    constexpr int per_cta = 2 * WPC;
    sqp_rows_kernel<NX, WPC><<<(a.ka.count + per_cta - 1) / per_cta, 32 * WPC, bytes, st>>>(a);
    return cudaGetLastError();
}

// a.ipc instances per CTA (0: 2)
template <int NX>
static cudaError_t launch_sqp_rows(const SqpArgs& a, cudaStream_t st)
{
    switch (a.ipc) {
        case 0:
        case 2: return launch_sqp_rows_w<NX, 1>(a, st);
        case 4: return launch_sqp_rows_w<NX, 2>(a, st);
        case 8: return launch_sqp_rows_w<NX, 4>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

// The scan fused SQP of small SRBD states with row-per-lane chunks: one
// instance per CTA, W chunks of 16 lanes (W / 2 warps).
template <int NX, int W>
static cudaError_t launch_sqp_scan_rows(const SqpArgs& a, cudaStream_t st)
{
    constexpr size_t bytes = ScanRowsSmem<NX, W>::BYTES;
    static_assert(bytes <= kSmemMax, "scan work areas fit shared memory");
    if (!a.lqcache) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> smem_done{0};
    if (cudaError_t e = ensure_smem(sqp_scan_rows_kernel<NX, W>, bytes, smem_done); e != cudaSuccess)
        return e;
    sqp_scan_rows_kernel<NX, W><<<a.ka.count, 16 * W, bytes, st>>>(a);
    return cudaGetLastError();
}

template <int NX, int NU>
static cudaError_t launch_sqp(const SqpArgs& a, int warps, cudaStream_t st)
{
    constexpr bool ROWS = NX == 12 && NU == 12;
    switch (warps) {
        case 1:
            if constexpr (ROWS) return launch_sqp_rows<NX>(a, st);
            else return launch_sqp_w<NX, NU, 1>(a, st);
        case 4:
            if constexpr (ROWS) return launch_sqp_scan_rows<NX, 4>(a, st);
            else return launch_sqp_w<NX, NU, 4>(a, st);
        case 8:
            if constexpr (ROWS) return launch_sqp_scan_rows<NX, 8>(a, st);
            else return launch_sqp_w<NX, NU, 8>(a, st);
        case 16:
            if constexpr (ROWS) return launch_sqp_scan_rows<NX, 16>(a, st);
            else return launch_sqp_w<NX, NU, 16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

// Dynamic shared memory of the fused kernel (its extras alone when the scan
// work areas live in the global workspace); SIZE_MAX when the warp count is
// not available for this size.
template <int NX, int NU, int W>
static size_t sqp_smem_w()
{
    using SM = SqpSmem<NX, NU, W>;
    if (W * UnitWarps<NX>::value * 32 > 1024) return SIZE_MAX;
    return SM::SC::BYTES > kSmemMax ? SM::EXTRA_BYTES : SM::BYTES;
}

template <int NX, int NU>
static size_t sqp_smem(int warps)
{
    constexpr bool ROWS = NX == 12 && NU == 12;
    switch (warps) {
        case 1:
            if constexpr (ROWS) return SqpRowsSmem<NX>::BYTES;
            else return sqp_smem_w<NX, NU, 1>();
        case 4:
            if constexpr (ROWS) return ScanRowsSmem<NX, 4>::BYTES;
            else return sqp_smem_w<NX, NU, 4>();
        case 8:
            if constexpr (ROWS) return ScanRowsSmem<NX, 8>::BYTES;
            else return sqp_smem_w<NX, NU, 8>();
        case 16:
            if constexpr (ROWS) return ScanRowsSmem<NX, 16>::BYTES;
            else return sqp_smem_w<NX, NU, 16>();
        default: return SIZE_MAX;
    }
}

template <int NX, int NU, bool SRBD = false, bool FUSED = false>
static SizeOps make_ops()
{
    SizeOps o{};
    o.n = NX;
    o.m = NU;
    o.scan = launch_scan<NX, NU>;
    o.riccati = launch_riccati<NX, NU>;
    o.resid = launch_resid<NX, NU>;
    o.scan_smem = scan_smem<NX, NU>;
    o.scan_checked = launch_scan_checked<NX, NU>;
    o.lq_stage_floats = StageL<NX, NU>::IN;
    o.scan_gws_floats = scan_gws_floats<NX, NU>;
    o.unit_warps = UnitWarps<NX>::value;
    if constexpr (UnitWarps<NX>::value == 8) {
        o.scan_split = launch_scan_split<NX, NU>;
        o.scan_split_gws_floats = scan_split_gws_floats<NX, NU>;
    }
    if constexpr (SRBD) {
        o.linearize = launch_linearize<NX, NU>;
        o.lin_ws_floats = lin_ws_floats<NX, NU>();
        o.merit = launch_merit<NX, NU>;
        o.sqp_step = launch_sqp_step<NX, NU>;
    }
    if constexpr (FUSED) {
        o.sqp = launch_sqp<NX, NU>;
        o.sqp_smem = sqp_smem<NX, NU>;
    }
    return o;
}


}  // namespace pdl
