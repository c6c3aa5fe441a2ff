// pdilqr.cu -- C ABI of the LQ KKT solvers (plans, validation, dispatch).
#include "pdilqr.h"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ops.h"
#include "plan.h"

using namespace pdl;

// ------------------------------------------------------------------ status
extern "C" const char* pdilqr_status_string(int s)
{
    switch (s) {
        case PDILQR_OK: return "ok";
        case PDILQR_E_INVALID_ARG: return "invalid argument";
        case PDILQR_E_NOT_SPD: return "matrix not positive definite";
        case PDILQR_E_SINGULAR: return "singular (I + C P) in a combine";
        case PDILQR_E_NONFINITE: return "non-finite value";
        case PDILQR_E_TIMEOUT: return "timeout";
        case PDILQR_E_NO_MEMORY: return "out of memory";
        case PDILQR_E_ADMISSION: return "admission refused";
        case PDILQR_E_LINESEARCH: return "line search found no step";
        case PDILQR_E_CUDA: return "CUDA error";
        default: return "unknown status";
    }
}

static pdilqr_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return PDILQR_OK;
    if (e == cudaErrorMemoryAllocation) return PDILQR_E_NO_MEMORY;
    return PDILQR_E_CUDA;
}
#define PD_CUDA(x)                                             \
    do {                                                       \
        cudaError_t e_ = (x);                                  \
        if (e_ != cudaSuccess) return cuda_status(e_);         \
    } while (0)

const SizeOps* pdl::find_ops(int n, int m)
{
    for (auto f : {ops_small, ops_12, ops_24, ops_36, ops_48, ops_96, ops_192})
        if (const SizeOps* o = f(n, m)) return o;
    return nullptr;
}

// -------------------------------------------------------------------- plan


static int pick_warps(const SizeOps* ops, int maxN)
{
    int w = maxN >= 40 ? 16 : (maxN >= 12 ? 8 : 4);
    while (w > 4 && (!warps_ok(ops, w) || ops->scan_smem(w) > kSmemMax)) w >>= 1;
    if (ops->scan_smem(w) > kSmemMax) {
        // global work areas; units wider than a warp take 4 chunks, which keeps
        // 128 registers per thread (the 1024-thread CTA of 8 such chunks spills)
        w = (maxN >= 40 && ops->unit_warps == 1) ? 8 : 4;
        while (w > 1 && !warps_ok(ops, w)) w >>= 1;
    }
    return w;
}

static pdilqr_status plan_init(pdilqr_plan* pl, const pdilqr_batch* b, const pdilqr_opts* o)
{
    pl->n = b->n;
    pl->m = b->m;
    pl->count = b->count;
    pl->ops = find_ops(b->n, b->m);
    if (!pl->ops) return PDILQR_E_INVALID_ARG;
    std::vector<int32_t> hN(b->N, b->N + b->count);
    std::vector<int64_t> hoff(b->stage_off, b->stage_off + b->count);
    // validate horizons and non-overlapping slot ranges
    std::vector<int32_t> by_off(b->count);
    for (int i = 0; i < b->count; ++i) {
        if (hN[i] < 1 || hN[i] > 4096 || hoff[i] < 0) return PDILQR_E_INVALID_ARG;
        by_off[i] = i;
        pl->maxN = std::max(pl->maxN, hN[i]);
        pl->total = std::max<int64_t>(pl->total, hoff[i] + hN[i] + 1);
    }
    std::sort(by_off.begin(), by_off.end(), [&](int x, int y) { return hoff[x] < hoff[y]; });
    for (int i = 1; i < b->count; ++i) {
        const int pa = by_off[i - 1], pb = by_off[i];
        if (hoff[pa] + hN[pa] + 1 > hoff[pb]) return PDILQR_E_INVALID_ARG;
    }
    pl->split = (o && o->split) ? 1 : 0;
    if (pl->split) {
        // chunks on separate CTAs: sizes with 8-warp units, 8 or 16 chunks
        if (!pl->ops->scan_split) return PDILQR_E_INVALID_ARG;
        pl->warps = (o && o->warps) ? o->warps : 16;
        if (pl->warps != 8 && pl->warps != 16) return PDILQR_E_INVALID_ARG;
    } else {
        pl->warps = (o && o->warps) ? o->warps : pick_warps(pl->ops, pl->maxN);
        if (!warps_ok(pl->ops, pl->warps)) return PDILQR_E_INVALID_ARG;
    }
    pl->refine = (o && o->refine) ? 1 : 0;
    // instances per CTA: only the row-per-lane sequential SQP (one-robot
    // SRBD, one chunk) packs several instances into a CTA
    pl->ipc = o ? o->inst_per_cta : 0;
    // FP64 elimination of the combines' M = I + C1 P2: the whole-body size
    pl->m64 = (o && o->m_fp64) ? 1 : 0;
    if (pl->m64 && !(pl->n == 36 && pl->m == 24)) return PDILQR_E_INVALID_ARG;
    if (pl->ipc != 0 && !(pl->n == 12 && pl->m == 12 && pl->warps == 1 &&
                          (pl->ipc == 2 || pl->ipc == 4 || pl->ipc == 8)))
        return PDILQR_E_INVALID_ARG;
    // longest horizons first: the tail of the grid holds the short instances
    std::vector<int32_t> order(b->count);
    for (int i = 0; i < b->count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hN[x] > hN[y]; });
    std::vector<int64_t> stage_inst(pl->total, -1);  // -1: slot of no instance
    for (int i = 0; i < b->count; ++i)
        for (int k = 0; k <= hN[i]; ++k) stage_inst[hoff[i] + k] = i;

    const size_t n = pl->n, m = pl->m, T = pl->total, C = pl->count;
    PD_CUDA(pl->alloc(&pl->dN, C));
    PD_CUDA(pl->alloc(&pl->doff, C));
    PD_CUDA(pl->alloc(&pl->dorder, C));
    PD_CUDA(pl->alloc(&pl->dstage_inst, T));
    PD_CUDA(pl->alloc(&pl->K, T * m * n));
    PD_CUDA(pl->alloc(&pl->k, T * m));
    PD_CUDA(pl->alloc(&pl->P, T * n * n));
    PD_CUDA(pl->alloc(&pl->p, T * n));
    PD_CUDA(pl->alloc(&pl->Abar, T * n * n));
    PD_CUDA(pl->alloc(&pl->bbar, T * n));
    PD_CUDA(pl->alloc(&pl->norms, C * 4));
    PD_CUDA(pl->alloc(&pl->st2, C));
    PD_CUDA(pl->alloc(&pl->rq, T * n));
    PD_CUDA(pl->alloc(&pl->rr, T * m));
    PD_CUDA(pl->alloc(&pl->rc, T * n));
    PD_CUDA(pl->alloc(&pl->rs, C * n));
    PD_CUDA(pl->alloc(&pl->ddx, T * n));
    PD_CUDA(pl->alloc(&pl->ddu, T * m));
    PD_CUDA(pl->alloc(&pl->ddl, T * n));
    // linearised-stage cache of the fused SQP (the one-chunk sweep linearises once)
    if (pl->ops->sqp && pl->warps > 1 && !pl->split)
        PD_CUDA(pl->alloc(&pl->lqcache, T * (size_t)pl->ops->lq_stage_floats));
    if (pl->split) {
        PD_CUDA(pl->alloc(&pl->gws, C * pl->ops->scan_split_gws_floats(pl->warps)));
        PD_CUDA(pl->alloc(&pl->sbar, C));
        if (pl->ops->sqp_step) {   // the unfused SQP iteration's buffers
            PD_CUDA(pl->alloc(&pl->lqA, T * n * n));
            PD_CUDA(pl->alloc(&pl->lqB, T * n * m));
            PD_CUDA(pl->alloc(&pl->lqc, T * n));
            PD_CUDA(pl->alloc(&pl->lqQ, T * n * n));
            PD_CUDA(pl->alloc(&pl->lqR, T * m * m));
            PD_CUDA(pl->alloc(&pl->lqq, T * n));
            PD_CUDA(pl->alloc(&pl->lqr, T * m));
            PD_CUDA(pl->alloc(&pl->sq_thmax, C));
            PD_CUDA(pl->alloc(&pl->sq_done, C));
            PD_CUDA(pl->alloc(&pl->sq_s, C * n));
        }
    } else if (const size_t gw = pl->ops->scan_gws_floats(pl->warps)) {
        PD_CUDA(pl->alloc(&pl->gws, C * gw));
    }
    if (pl->ops->lin_ws_floats) PD_CUDA(pl->alloc(&pl->lin_ws, pl->ops->lin_ws_floats));
    PD_CUDA(cudaMemcpy(pl->dN, hN.data(), C * sizeof(int32_t), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(pl->doff, hoff.data(), C * sizeof(int64_t), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(pl->dorder, order.data(), C * sizeof(int32_t), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(pl->dstage_inst, stage_inst.data(), T * sizeof(int64_t),
                       cudaMemcpyHostToDevice));
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_plan_create(const pdilqr_batch* b, const pdilqr_opts* o,
                                            pdilqr_plan** out)
{
    if (!out) return PDILQR_E_INVALID_ARG;
    *out = nullptr;
    if (!b || !b->N || !b->stage_off || b->count < 1 || b->n < 1 || b->m < 1)
        return PDILQR_E_INVALID_ARG;
    pdilqr_plan* pl = new (std::nothrow) pdilqr_plan();
    if (!pl) return PDILQR_E_NO_MEMORY;
    pdilqr_status st = plan_init(pl, b, o);
    if (st != PDILQR_OK) {
        delete pl;
        return st;
    }
    *out = pl;
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_plan_destroy(pdilqr_plan* pl)
{
    delete pl;
    return PDILQR_OK;
}

extern "C" int32_t pdilqr_plan_warps(const pdilqr_plan* pl) { return pl ? pl->warps : 0; }

extern "C" pdilqr_status pdilqr_plan_set_debug(pdilqr_plan* pl, int32_t flags)
{
    if (!pl || (flags & ~(PDILQR_DEBUG_TC_SKIP_ISSUE | PDILQR_DEBUG_BULK_SKIP_ISSUE |
                          PDILQR_DEBUG_SPLIT_SKIP_ARRIVE)))
        return PDILQR_E_INVALID_ARG;
    pl->dbg = flags;
    return PDILQR_OK;
}

// ------------------------------------------------------------- KKT solves
static KktArgs make_args(pdilqr_plan* pl, const pdilqr_lq* lq, const float* s, float* dx,
                         float* du, float* dl, float* K, float* k, float* P, float* p,
                         int32_t* status)
{
    KktArgs a;
    a.A = lq->A; a.B = lq->B; a.c = lq->c; a.Q = lq->Q; a.R = lq->R; a.S = lq->S;
    a.q = lq->q; a.r = lq->r;
    a.s = s;
    a.dx = dx; a.du = du; a.dlam = dl;
    a.K = K ? K : pl->K;
    a.k = k ? k : pl->k;
    a.P = P ? P : pl->P;
    a.p = p ? p : pl->p;
    a.Abar = pl->Abar;
    a.bbar = pl->bbar;
    a.N = pl->dN;
    a.off = pl->doff;
    a.order = pl->dorder;
    a.status = status;
    a.count = pl->count;
    a.gws = pl->gws;
    a.m64 = pl->m64;
    a.sbar = pl->sbar;
    a.dbg = pl->dbg;
    return a;
}

// Every per-stage array is read (and the policy outputs written) with 16-byte
// accesses: a misaligned pointer is an invalid argument, not a fault.
static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static bool lq_ok(const pdilqr_lq* lq)
{
    return lq && lq->A && lq->B && lq->c && lq->Q && lq->R && lq->q && lq->r &&
           aligned16(lq->A) && aligned16(lq->B) && aligned16(lq->c) && aligned16(lq->Q) &&
           aligned16(lq->R) && aligned16(lq->q) && aligned16(lq->r) && aligned16(lq->S);
}

static pdilqr_status residual_into(pdilqr_plan* pl, const pdilqr_lq* lq, const float* s,
                                   const float* dx, const float* du, const float* dl,
                                   double* norms, bool want_rhs, cudaStream_t st)
{
    PD_CUDA(cudaMemsetAsync(norms, 0, sizeof(double) * 4 * pl->count, st));
    ResidArgs r;
    r.A = lq->A; r.B = lq->B; r.c = lq->c; r.Q = lq->Q; r.R = lq->R; r.S = lq->S;
    r.q = lq->q; r.r = lq->r; r.s = s;
    r.dx = dx; r.du = du; r.dlam = dl;
    r.N = pl->dN;
    r.off = pl->doff;
    r.stage_inst = pl->dstage_inst;
    r.total_stages = pl->total;
    r.norms = norms;
    r.rq = want_rhs ? pl->rq : nullptr;
    r.rr = want_rhs ? pl->rr : nullptr;
    r.rc = want_rhs ? pl->rc : nullptr;
    r.rs = want_rhs ? pl->rs : nullptr;
    PD_CUDA(pl->ops->resid(r, st));
    return PDILQR_OK;
}

// status[i] = max(status[i], st2[i]): the correction solve's verdict joins the first one's
__global__ void status_merge_kernel(int32_t* status, const int32_t* st2, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && st2[i] > status[i]) status[i] = st2[i];
}

static cudaError_t launch_axpy(float* z, const float* dz, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    axpy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(z, dz, n);
    return cudaGetLastError();
}

static pdilqr_status solve_common(pdilqr_plan* pl, const pdilqr_lq* lq, const float* s,
                                  pdilqr_kkt_out* out, cudaStream_t st, bool scan)
{
    if (!pl || !lq_ok(lq) || !s || !out || !out->dx || !out->du || !out->dlam || !out->status)
        return PDILQR_E_INVALID_ARG;
    if (!aligned16(out->K) || !aligned16(out->k) || !aligned16(out->P) || !aligned16(out->p))
        return PDILQR_E_INVALID_ARG;
    if (scan && pl->ops->scan_smem(pl->warps) > kSmemMax && !pl->gws) return PDILQR_E_INVALID_ARG;
    auto run = [&](const KktArgs& a) -> cudaError_t {
        if (!scan) return pl->ops->riccati(a, st);
        return pl->split ? pl->ops->scan_split(a, pl->warps, st) : pl->ops->scan(a, pl->warps, st);
    };
    KktArgs a = make_args(pl, lq, s, out->dx, out->du, out->dlam, out->K, out->k, out->P,
                          out->p, out->status);
    PD_CUDA(run(a));
    if (pl->refine) {
        // one correction solve against the FP64 residual
        pdilqr_status rs = residual_into(pl, lq, s, out->dx, out->du, out->dlam, pl->norms,
                                         true, st);
        if (rs != PDILQR_OK) return rs;
        pdilqr_lq corr = {lq->A, lq->B, pl->rc, lq->Q, lq->R, lq->S, pl->rq, pl->rr};
        KktArgs b = make_args(pl, &corr, pl->rs, pl->ddx, pl->ddu, pl->ddl, nullptr, nullptr,
                              nullptr, nullptr, pl->st2);
        PD_CUDA(run(b));
        status_merge_kernel<<<(pl->count + 255) / 256, 256, 0, st>>>(out->status, pl->st2, pl->count);
        PD_CUDA(cudaGetLastError());
        const int64_t T = pl->total;
        PD_CUDA(launch_axpy(out->dx, pl->ddx, T * pl->n, st));
        PD_CUDA(launch_axpy(out->du, pl->ddu, T * pl->m, st));
        PD_CUDA(launch_axpy(out->dlam, pl->ddl, T * pl->n, st));
        if (out->k) PD_CUDA(launch_axpy(out->k, pl->k, T * pl->m, st));
        if (out->p) PD_CUDA(launch_axpy(out->p, pl->p, T * pl->n, st));
    }
    if (out->resid) {
        pdilqr_status rs = residual_into(pl, lq, s, out->dx, out->du, out->dlam, out->resid,
                                         false, st);
        if (rs != PDILQR_OK) return rs;
    }
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_kkt_scan_solve(pdilqr_plan* pl, const pdilqr_lq* lq,
                                               const float* s, pdilqr_kkt_out* out,
                                               pdilqr_stream stream)
{
    return solve_common(pl, lq, s, out, (cudaStream_t)stream, true);
}

extern "C" pdilqr_status pdilqr_riccati_solve(pdilqr_plan* pl, const pdilqr_lq* lq,
                                              const float* s, pdilqr_kkt_out* out,
                                              pdilqr_stream stream)
{
    return solve_common(pl, lq, s, out, (cudaStream_t)stream, false);
}

extern "C" pdilqr_status pdilqr_kkt_residual(pdilqr_plan* pl, const pdilqr_lq* lq,
                                             const float* s, const float* dx, const float* du,
                                             const float* dlam, double* resid,
                                             pdilqr_stream stream)
{
    if (!pl || !lq_ok(lq) || !s || !dx || !du || !dlam || !resid) return PDILQR_E_INVALID_ARG;
    return residual_into(pl, lq, s, dx, du, dlam, resid, false, (cudaStream_t)stream);
}

// ------------------------------------------------------------ SRBD model
static bool model_ok(const pdilqr_plan* pl, const pdilqr_srbd_model* md)
{
    return md && md->nrob >= 1 && md->nrob <= 16 && pl->n == 12 * md->nrob && pl->m == pl->n &&
           md->dt > 0.f && md->mass > 0.f && md->inertia[0] > 0.f && md->inertia[1] > 0.f &&
           md->inertia[2] > 0.f && md->bar_delta > 0.f;
}

extern "C" pdilqr_status pdilqr_linearize(pdilqr_plan* pl, const pdilqr_srbd_model* md,
                                          const pdilqr_traj* tr, pdilqr_lq_out* out,
                                          pdilqr_stream stream)
{
    if (!pl || !model_ok(pl, md) || !pl->ops->linearize || !tr || !out) return PDILQR_E_INVALID_ARG;
    if (!tr->x || !tr->u || !tr->lam || !tr->xref || !tr->uref || !tr->contact)
        return PDILQR_E_INVALID_ARG;
    if (!out->A || !out->B || !out->c || !out->Q || !out->R || !out->q || !out->r)
        return PDILQR_E_INVALID_ARG;
    LinArgs a;
    a.md = *md;
    a.x = tr->x; a.u = tr->u; a.lam = tr->lam; a.xref = tr->xref; a.uref = tr->uref;
    a.contact = tr->contact;
    a.A = out->A; a.B = out->B; a.c = out->c; a.Q = out->Q; a.R = out->R; a.S = out->S;
    a.q = out->q; a.r = out->r;
    a.N = pl->dN;
    a.off = pl->doff;
    a.stage_inst = pl->dstage_inst;
    a.total = pl->total;
    a.work = pl->lin_ws;
    PD_CUDA(pl->ops->linearize(a, (cudaStream_t)stream));
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_merit_eval(pdilqr_plan* pl, const pdilqr_srbd_model* md,
                                           const pdilqr_traj* tr, const float* x0hat,
                                           const float* dx, const float* du, double* merit,
                                           pdilqr_stream stream)
{
    if (!pl || !model_ok(pl, md) || !pl->ops->merit || !tr || !x0hat || !dx || !du || !merit)
        return PDILQR_E_INVALID_ARG;
    if (!tr->x || !tr->u || !tr->xref || !tr->uref || !tr->contact) return PDILQR_E_INVALID_ARG;
    MeritArgs a;
    a.md = *md;
    a.x = tr->x; a.u = tr->u; a.xref = tr->xref; a.uref = tr->uref; a.x0hat = x0hat;
    a.dx = dx; a.du = du; a.contact = tr->contact;
    a.N = pl->dN;
    a.off = pl->doff;
    a.out = merit;
    a.count = pl->count;
    PD_CUDA(pl->ops->merit(a, (cudaStream_t)stream));
    return PDILQR_OK;
}

// The SQP of a split plan (the scan's chunks on separate CTAs): an unfused
// iteration per SQP step (Sec. II-B..II-E), all on the stream -- the
// linearisation of every stage into the plan's LQ arrays, the split scan of
// the KKT system (dx_0 from the step kernel), and the step kernel (merit of
// the ten step sizes, filter decision, update, next dx_0).  Instances that
// have stopped are skipped by the step kernel; their stages are still
// linearised and solved by later iterations (the launches are uniform).
static pdilqr_status solve_split(pdilqr_plan* pl, const pdilqr_srbd_model* md,
                                 const pdilqr_sqp_opts* o, const float* x0hat, float* x, float* u,
                                 float* lam, const float* xref, const float* uref,
                                 const uint8_t* contact, pdilqr_sqp_info* info, cudaStream_t st)
{
    if (!pl->ops->sqp_step || !pl->lqA || !pl->ops->linearize) return PDILQR_E_INVALID_ARG;
    LinArgs la;
    la.md = *md;
    la.x = x; la.u = u; la.lam = lam; la.xref = xref; la.uref = uref; la.contact = contact;
    la.A = pl->lqA; la.B = pl->lqB; la.c = pl->lqc; la.Q = pl->lqQ; la.R = pl->lqR; la.S = nullptr;
    la.q = pl->lqq; la.r = pl->lqr;
    la.N = pl->dN;
    la.off = pl->doff;
    la.stage_inst = pl->dstage_inst;
    la.total = pl->total;
    la.work = pl->lin_ws;
    const pdilqr_lq lq = {pl->lqA, pl->lqB, pl->lqc, pl->lqQ, pl->lqR, nullptr, pl->lqq, pl->lqr};
    const KktArgs ka = make_args(pl, &lq, pl->sq_s, pl->ddx, pl->ddu, pl->ddl, nullptr, nullptr,
                                 nullptr, nullptr, pl->st2);
    SqpStepArgs sa;
    sa.md = *md;
    sa.x0hat = x0hat;
    sa.x = x; sa.u = u; sa.lam = lam; sa.xref = xref; sa.uref = uref; sa.contact = contact;
    sa.dx = pl->ddx; sa.du = pl->ddu; sa.dlam = pl->ddl;
    sa.N = pl->dN;
    sa.off = pl->doff;
    sa.count = pl->count;
    sa.max_iters = o->max_iters;
    sa.tol_step = o->tol_step;
    sa.tol_theta = o->tol_theta;
    sa.c_armijo = o->c_armijo;
    sa.theta_frac = o->theta_frac;
    sa.alpha_replay = o->alpha_replay;
    sa.iters = info->iters;
    sa.status = info->status;
    sa.alpha = info->alpha;
    sa.J = info->J;
    sa.theta = info->theta;
    sa.kst = pl->st2;
    sa.thmax = pl->sq_thmax;
    sa.done = pl->sq_done;
    sa.s = pl->sq_s;
    sa.it = -1;
    PD_CUDA(pl->ops->sqp_step(sa, st));
    for (int it = 0; it < o->max_iters; ++it) {
        PD_CUDA(pl->ops->linearize(la, st));
        PD_CUDA(pl->ops->scan_split(ka, pl->warps, st));
        sa.it = it;
        PD_CUDA(pl->ops->sqp_step(sa, st));
    }
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_solve(pdilqr_plan* pl, const pdilqr_srbd_model* md,
                                      const pdilqr_sqp_opts* o, const float* x0hat, float* x,
                                      float* u, float* lam, const float* xref, const float* uref,
                                      const uint8_t* contact, pdilqr_sqp_info* info,
                                      pdilqr_stream stream)
{
    if (!pl || !model_ok(pl, md) || !pl->ops->sqp || !o || !info) return PDILQR_E_INVALID_ARG;
    if (!x0hat || !x || !u || !lam || !xref || !uref || !contact || !info->iters || !info->status)
        return PDILQR_E_INVALID_ARG;
    if (o->max_iters < 1 || o->max_iters > 32) return PDILQR_E_INVALID_ARG;
    if (pl->split) return solve_split(pl, md, o, x0hat, x, u, lam, xref, uref, contact, info,
                                      (cudaStream_t)stream);
    if (pl->ops->sqp_smem(pl->warps) > kSmemMax) return PDILQR_E_INVALID_ARG;
    if (pl->ops->scan_gws_floats(pl->warps) && !pl->gws) return PDILQR_E_INVALID_ARG;
    SqpArgs a;
    a.md = *md;
    a.x0hat = x0hat;
    a.x = x; a.u = u; a.lam = lam; a.xref = xref; a.uref = uref; a.contact = contact;
    pdilqr_lq none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    a.ka = make_args(pl, &none, nullptr, pl->ddx, pl->ddu, pl->ddl, nullptr, nullptr, nullptr,
                     nullptr, pl->st2);
    a.max_iters = o->max_iters;
    a.tol_step = o->tol_step;
    a.tol_theta = o->tol_theta;
    a.c_armijo = o->c_armijo;
    a.theta_frac = o->theta_frac;
    a.alpha_replay = o->alpha_replay;
    a.iters = info->iters;
    a.status = info->status;
    a.alpha = info->alpha;
    a.J = info->J;
    a.theta = info->theta;
    a.lqcache = pl->lqcache;
    a.ipc = pl->ipc;
    PD_CUDA(pl->ops->sqp(a, pl->warps, (cudaStream_t)stream));
    return PDILQR_OK;
}

// ------------------------------------------------------ captured solves
extern "C" pdilqr_status pdilqr_solve_capture(pdilqr_plan* pl, const pdilqr_srbd_model* md,
                                              const pdilqr_sqp_opts* o, const float* x0hat,
                                              float* x, float* u, float* lam, const float* xref,
                                              const float* uref, const uint8_t* contact,
                                              pdilqr_sqp_info* info)
{
    if (!pl || pl->split) return PDILQR_E_INVALID_ARG;   // split plans: direct solves only
    cudaStream_t s = nullptr;
    PD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return cuda_status(e);
    }
    const pdilqr_status st = pdilqr_solve(pl, md, o, x0hat, x, u, lam, xref, uref, contact, info,
                                          (pdilqr_stream)s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);   // ends the capture whatever the solve returned
    cudaStreamDestroy(s);
    if (st != PDILQR_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_status(e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e);
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    pl->graph = ex;
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_plan_replay(pdilqr_plan* pl, pdilqr_stream stream)
{
    if (!pl || !pl->graph) return PDILQR_E_INVALID_ARG;
    PD_CUDA(cudaGraphLaunch(pl->graph, (cudaStream_t)stream));
    return PDILQR_OK;
}

// ------------------------------------------------ allocation-free scan solve
// Scratch of pdilqr_kkt_scan_solve_noalloc: a file-scope device array that
// every GPU loading this library holds until the process exits.  Host code
// must not hand the array's name to a kernel (on the host it only stands in
// for the symbol); the device address is looked up once per device.
static constexpr size_t kNoAllocFloats = size_t(4) << 20;  // 16 MiB
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

static std::mutex g_noalloc_mu;
static float* g_noalloc_addr[64] = {};

static pdilqr_status noalloc_base(float** out)
{
    int dev = -1;
    PD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return PDILQR_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return e != cudaSuccess ? cuda_status(e) : PDILQR_E_CUDA;
        g_noalloc_addr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_addr[dev];
    return PDILQR_OK;
}

extern "C" int64_t pdilqr_noalloc_capacity_stages(int32_t n, int32_t m)
{
    if (n < 1 || m < 1) return 0;
    const size_t per = (size_t)m * n + m + 2 * (size_t)n * n + 2 * (size_t)n;
    // six regions, each rounded up to 64 floats
    return (int64_t)((kNoAllocFloats - 6 * 64) / per);
}

extern "C" pdilqr_status pdilqr_kkt_scan_solve_noalloc(
    int32_t n, int32_t m, int32_t count, int64_t total_stages, const int32_t* N,
    const int64_t* stage_off, int32_t warps, const pdilqr_lq* lq, const float* s, float* dx,
    float* du, float* dlam, int32_t* status, pdilqr_stream stream)
{
    const SizeOps* ops = find_ops(n, m);
    if (!ops || count < 1 || total_stages < 2 || !N || !stage_off || !lq_ok(lq) || !s || !dx ||
        !du || !dlam || !status)
        return PDILQR_E_INVALID_ARG;
    if (total_stages > pdilqr_noalloc_capacity_stages(n, m)) return PDILQR_E_INVALID_ARG;
    if (warps == 0) warps = 8;
    if (warps != 4 && warps != 8 && warps != 16) return PDILQR_E_INVALID_ARG;
    if (ops->scan_smem(warps) > kSmemMax) return PDILQR_E_INVALID_ARG;
    float* base = nullptr;
    pdilqr_status st = noalloc_base(&base);
    if (st != PDILQR_OK) return st;
    auto region = [&](size_t floats_per_stage) {
        float* r = base;
        base += (((size_t)total_stages * floats_per_stage) + 63) / 64 * 64;
        return r;
    };
    KktArgs a;
    a.A = lq->A; a.B = lq->B; a.c = lq->c; a.Q = lq->Q; a.R = lq->R; a.S = lq->S;
    a.q = lq->q; a.r = lq->r;
    a.s = s;
    a.dx = dx; a.du = du; a.dlam = dlam;
    a.K = region((size_t)m * n);
    a.k = region((size_t)m);
    a.P = region((size_t)n * n);
    a.p = region((size_t)n);
    a.Abar = region((size_t)n * n);
    a.bbar = region((size_t)n);
    a.N = N;
    a.off = stage_off;
    a.order = nullptr;
    a.status = status;
    a.count = count;
    a.gws = nullptr;
    a.dbg = 0;
    PD_CUDA(ops->scan_checked(a, warps, total_stages, (cudaStream_t)stream));
    return PDILQR_OK;
}

// ------------------------------------------------------------ capacity plans
pdilqr_status pdl::plan_create_capacity(int n, int m, int max_count, int64_t slots, int warps,
                                        pdilqr_plan** out)
{
    *out = nullptr;
    const SizeOps* ops = find_ops(n, m);
    if (!ops || max_count < 1 || slots < 2 || !warps_ok(ops, warps)) return PDILQR_E_INVALID_ARG;
    pdilqr_plan* pl = new (std::nothrow) pdilqr_plan();
    if (!pl) return PDILQR_E_NO_MEMORY;
    pl->n = n;
    pl->m = m;
    pl->ops = ops;
    pl->count = 0;
    pl->max_count = max_count;
    pl->total = slots;
    pl->warps = warps;
    const size_t T = slots, C = max_count;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    chk(pl->alloc(&pl->dN, C));
    chk(pl->alloc(&pl->doff, C));
    chk(pl->alloc(&pl->dorder, C));
    chk(pl->alloc(&pl->dstage_inst, T));
    chk(pl->alloc(&pl->K, T * m * n));
    chk(pl->alloc(&pl->k, T * m));
    chk(pl->alloc(&pl->P, T * n * n));
    chk(pl->alloc(&pl->p, T * n));
    chk(pl->alloc(&pl->Abar, T * n * n));
    chk(pl->alloc(&pl->bbar, T * n));
    chk(pl->alloc(&pl->norms, C * 4));
    chk(pl->alloc(&pl->st2, C));
    chk(pl->alloc(&pl->ddx, T * n));
    chk(pl->alloc(&pl->ddu, T * m));
    chk(pl->alloc(&pl->ddl, T * n));
    if (ops->sqp && warps > 1) chk(pl->alloc(&pl->lqcache, T * (size_t)ops->lq_stage_floats));
    if (const size_t gw = ops->scan_gws_floats(warps)) chk(pl->alloc(&pl->gws, C * gw));
    if (e != cudaSuccess) {
        delete pl;
        return cuda_status(e);
    }
    *out = pl;
    return PDILQR_OK;
}

pdilqr_status pdl::plan_enable_split(pdilqr_plan* pl, int warps)
{
    if (!pl || pl->split || pl->warps != 1 || (warps != 8 && warps != 16)) return PDILQR_E_INVALID_ARG;
    const SizeOps* ops = pl->ops;
    if (!ops->scan_split || !ops->sqp_step || !ops->linearize) return PDILQR_E_INVALID_ARG;
    const size_t n = pl->n, m = pl->m, T = pl->total, C = pl->max_count;
    PD_CUDA(pl->alloc(&pl->gws, C * ops->scan_split_gws_floats(warps)));
    PD_CUDA(pl->alloc(&pl->sbar, C));
    PD_CUDA(pl->alloc(&pl->lqA, T * n * n));
    PD_CUDA(pl->alloc(&pl->lqB, T * n * m));
    PD_CUDA(pl->alloc(&pl->lqc, T * n));
    PD_CUDA(pl->alloc(&pl->lqQ, T * n * n));
    PD_CUDA(pl->alloc(&pl->lqR, T * m * m));
    PD_CUDA(pl->alloc(&pl->lqq, T * n));
    PD_CUDA(pl->alloc(&pl->lqr, T * m));
    PD_CUDA(pl->alloc(&pl->sq_thmax, C));
    PD_CUDA(pl->alloc(&pl->sq_done, C));
    PD_CUDA(pl->alloc(&pl->sq_s, C * n));
    if (ops->lin_ws_floats && !pl->lin_ws) PD_CUDA(pl->alloc(&pl->lin_ws, ops->lin_ws_floats));
    pl->warps = warps;
    pl->split = 1;
    return PDILQR_OK;
}

pdilqr_status pdl::plan_set_stage_inst_async(pdilqr_plan* pl, const int64_t* hstage, cudaStream_t st)
{
    if (!pl || !hstage) return PDILQR_E_INVALID_ARG;
    PD_CUDA(cudaMemcpyAsync(pl->dstage_inst, hstage, sizeof(int64_t) * pl->total,
                            cudaMemcpyHostToDevice, st));
    return PDILQR_OK;
}

pdilqr_status pdl::plan_set_batch_async(pdilqr_plan* pl, const int32_t* hN, const int64_t* hoff,
                                        const int32_t* horder, int count, int maxN, cudaStream_t st)
{
    if (count < 1 || count > pl->max_count) return PDILQR_E_INVALID_ARG;
    PD_CUDA(cudaMemcpyAsync(pl->dN, hN, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
    PD_CUDA(cudaMemcpyAsync(pl->doff, hoff, sizeof(int64_t) * count, cudaMemcpyHostToDevice, st));
    PD_CUDA(cudaMemcpyAsync(pl->dorder, horder, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
    pl->count = count;
    pl->maxN = maxN;
    return PDILQR_OK;
}
