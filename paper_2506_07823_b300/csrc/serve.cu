// serve.cu -- continuous-batching MPC server around the fused SQP kernel.
//
// Clients hold their warm start (x, u, lam) and references on the device in
// blocks carved from one pool.  A dispatcher thread forms batches from the
// pending requests whose clients are idle (one size class per batch), and
// for each batch, on one of several streams:
//   1. copies the staged request data (x0hat, new references) to the device,
//   2. gathers every client's state into packed batch arrays, shifted by one
//      step (the real-time-iteration warm start) unless the client is new,
//   3. runs pdilqr_solve on the packed batch,
//   4. scatters the solution back into the client blocks and copies the
//      trajectories and status words to pinned host memory,
//   5. signals completion through a host callback.
// Batches on different streams run concurrently; a client is never in two
// batches at once.  Every wait is bounded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.h"

using namespace pdl;
using Clock = std::chrono::steady_clock;

namespace {

// size classes nrob = 1, 2, 4, 8, 16 (class c holds 2^c robots, n = m = 12 nrob)
constexpr int kClasses = 5;

int class_of(int nrob)
{
    for (int c = 0; c < kClasses; ++c)
        if (nrob == (1 << c)) return c;
    return -1;
}

struct Entry {  // one request of a launch (device table)
    float *cx, *cu, *cl, *cxr, *cur;
    uint8_t* cct;
    int64_t off;    // first packed stage slot
    int64_t soff;   // first staged reference slot (when refs != 0)
    int32_t N, init, refs, pad;
};

__global__ void serve_gather(const Entry* tab, int n, int nc, const float* __restrict__ sxr,
                             const float* __restrict__ sur, const uint8_t* __restrict__ sct,
                             const float* __restrict__ x0, float* px, float* pu, float* pl,
                             float* pxr, float* pur, uint8_t* pct)
{
    const Entry e = tab[blockIdx.x];
    const int N = e.N;
    for (int idx = threadIdx.x; idx < (N + 1) * n; idx += blockDim.x) {
        const int k = idx / n, i = idx % n;
        const int64_t dst = (e.off + k) * n + i;
        const int ks = min(k + 1, N);          // shifted state / costate slot
        const int ku = min(k + 1, N - 1);      // shifted control slot
        float xr, ur;
        if (e.refs) {
            xr = sxr[(e.soff + k) * n + i];
            ur = sur[(e.soff + k) * n + i];
        } else {
            xr = e.cxr[(int64_t)ks * n + i];
            ur = e.cur[(int64_t)ku * n + i];
        }
        pxr[dst] = xr;
        pur[dst] = k < N ? ur : 0.f;
        if (e.init) {
            px[dst] = x0[(int64_t)blockIdx.x * n + i];
            pu[dst] = k < N ? ur : 0.f;
            pl[dst] = 0.f;
        } else {
            px[dst] = e.cx[(int64_t)ks * n + i];
            pu[dst] = k < N ? e.cu[(int64_t)ku * n + i] : 0.f;
            pl[dst] = e.cl[(int64_t)ks * n + i];
        }
    }
    for (int idx = threadIdx.x; idx < (N + 1) * nc; idx += blockDim.x) {
        const int k = idx / nc, j = idx % nc;
        pct[(e.off + k) * nc + j] =
            e.refs ? sct[(e.soff + k) * nc + j] : e.cct[(int64_t)min(k + 1, N) * nc + j];
    }
}

__global__ void serve_scatter(const Entry* tab, int n, int nc, const float* px, const float* pu,
                              const float* pl, const float* pxr, const float* pur,
                              const uint8_t* pct)
{
    const Entry e = tab[blockIdx.x];
    const int N = e.N;
    for (int idx = threadIdx.x; idx < (N + 1) * n; idx += blockDim.x) {
        const int64_t src = e.off * n + idx;
        e.cx[idx] = px[src];
        e.cu[idx] = pu[src];
        e.cl[idx] = pl[src];
        e.cxr[idx] = pxr[src];
        e.cur[idx] = pur[src];
    }
    for (int idx = threadIdx.x; idx < (N + 1) * nc; idx += blockDim.x) e.cct[idx] = pct[e.off * nc + idx];
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Client {
    int nrob = 0, n = 0, N = 0;
    size_t off = 0, bytes = 0;
    bool busy = false, has_state = false;
    float *x, *u, *l, *xr, *ur;
    uint8_t* ct;
};

struct Request {
    uint64_t ticket, client;
    int nrob, N, reset;
    bool refs;
    std::vector<float> x0, xr, ur;
    std::vector<uint8_t> ct;
    Clock::time_point t0;
};

struct Result {
    Clock::time_point t0;
    bool done = false;
    int32_t status = 0, iters = 0;
    int64_t latency_ns = 0;
    int n = 0, N = 0;
    std::vector<float> x, u;
};

struct ClassRes {  // device and pinned buffers of one size class on one stream
    bool ready = false;
    int n = 0, nc = 0;
    pdilqr_plan* plan = nullptr;
    float *px, *pu, *pl, *pxr, *pur, *px0, *sxr, *sur;
    uint8_t *pct, *sct;
    int32_t *dit, *dst;
    Entry* dtab;
    // pinned
    Entry* htab;
    int32_t *hN, *horder, *hit, *hst;
    int64_t* hoff;
    int64_t* hstage = nullptr;   // stage slot -> instance (split classes)
    int64_t slots = 0;           // stage slots of the capacity plan
    float *hx0, *hxr, *hur, *hxo, *huo;
    uint8_t* hct;
    std::vector<void*> dev, host;
};

struct Slot {  // one stream with its batch
    cudaStream_t s = nullptr;
    bool busy = false, done = false;
    int cls = 0, count = 0;
    std::vector<uint64_t> tickets, clients;
    std::vector<int64_t> offs;
    std::vector<int> Ns;
    ClassRes res[kClasses];
};

class Pool {  // first-fit allocator over [0, total) in 256-byte units
public:
    void init(size_t total) { free_.clear(); free_[0] = total; total_ = total; used_ = 0; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t total() const { return total_; }

private:
    std::map<size_t, size_t> free_;
    size_t total_ = 0, used_ = 0;
};

}  // namespace

struct pdilqr_server {
    pdilqr_serve_opts opts{};
    pdilqr_srbd_model models[kClasses];   // constants per size class
    int device = 0;
    uint8_t* pool_base = nullptr;
    Pool pool;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::unordered_map<uint64_t, Client> clients;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Result> results;
    std::vector<Slot> slots;
    // statistics
    int64_t submitted = 0, completed = 0, refused = 0, batches = 0, batched_requests = 0;
    bool class_admitted[5] = {false, false, false, false, false};   // free-memory check passed
    bool started = false;
    Clock::time_point t_first;
    std::vector<int64_t> lat;   // ring of recent latencies (ns)
    size_t lat_pos = 0;
};

namespace {

constexpr size_t kLatRing = 1 << 17;

size_t client_bytes(int nrob, int N)
{
    const size_t n = 12 * (size_t)nrob, S = (size_t)N + 1;
    return 5 * align256(S * n * sizeof(float)) + align256(S * 4 * nrob);
}

void carve_client(pdilqr_server* sv, Client& c)
{
    const size_t S = (size_t)c.N + 1, fb = align256(S * c.n * sizeof(float));
    uint8_t* b = sv->pool_base + c.off;
    c.x = reinterpret_cast<float*>(b);
    c.u = reinterpret_cast<float*>(b + fb);
    c.l = reinterpret_cast<float*>(b + 2 * fb);
    c.xr = reinterpret_cast<float*>(b + 3 * fb);
    c.ur = reinterpret_cast<float*>(b + 4 * fb);
    c.ct = b + 5 * fb;
}

template <typename T>
cudaError_t dalloc(ClassRes& r, T** p, size_t count)
{
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) { r.dev.push_back(v); *p = static_cast<T*>(v); }
    return e;
}

template <typename T>
cudaError_t halloc(ClassRes& r, T** p, size_t count)
{
    void* v = nullptr;
    cudaError_t e = cudaHostAlloc(&v, std::max<size_t>(count, 1) * sizeof(T), cudaHostAllocDefault);
    if (e == cudaSuccess) { r.host.push_back(v); *p = static_cast<T*>(v); }
    return e;
}

void free_res(ClassRes& r)
{
    if (r.plan) pdilqr_plan_destroy(r.plan);
    for (void* v : r.dev) cudaFree(v);
    for (void* v : r.host) cudaFreeHost(v);
    r = ClassRes{};
}

// Largest batch of size class cls (2^cls robots): the configured maximum for
// one robot, a quarter of it per doubling of the robot count (the per-stage
// workspace grows with n^2), at least 64.
int class_batch(const pdilqr_server* sv, int cls)
{
    const int b = std::max(64, sv->opts.max_batch >> (2 * cls));
    return std::min(b, sv->opts.max_batch);
}

// Classes of four or more robots run for tens of milliseconds per batch; with
// more than one stream they may hold all but one, which stays free for the
// one- and two-robot classes.
constexpr int kLargeClass = 2;

// Horizon chunks (CTAs) per instance of a split class.
constexpr int kSplitChunks = 16;

// Whether size class cls runs a split plan (the server's split_min_robots).
bool class_split(const pdilqr_server* sv, int cls)
{
    return sv->opts.split_min_robots > 0 && (1 << cls) >= sv->opts.split_min_robots;
}

// Largest batch of size class cls as launched: a split class is also capped
// by split_max_batch (each instance holds kSplitChunks SMs while it runs).
int class_cap(const pdilqr_server* sv, int cls)
{
    const int b = class_batch(sv, cls);
    return class_split(sv, cls) ? std::min(b, sv->opts.split_max_batch) : b;
}

// Device bytes of one stream's batch workspace for size class cls: the
// capacity plan (policy, value function and closed-loop maps per stage slot,
// the step buffers, the linearised-stage cache of the scan) and the staging
// arrays ensure_res allocates.
size_t class_res_bytes(const pdilqr_server* sv, int cls)
{
    const int nrob = 1 << cls;
    const size_t n = 12 * (size_t)nrob, B = class_cap(sv, cls);
    const size_t S = B * ((size_t)sv->opts.max_N + 1);
    const SizeOps* ops = find_ops((int)n, (int)n);
    const bool split = class_split(sv, cls);
    // a split plan keeps the linearised LQ arrays (A, B, Q, R, c, q, r) and the
    // stage map instead of the stage cache, and a chunk work area per CTA
    const size_t lq = split ? 4 * n * n + 5 * n : (ops ? (size_t)ops->lq_stage_floats : 0);
    const size_t per_slot = 3 * n * n + 6 * n + lq + 8 * n + 4 * nrob;
    const size_t gws = (split && ops && ops->scan_split_gws_floats)
                           ? ops->scan_split_gws_floats(kSplitChunks) : 0;
    return sizeof(float) * S * per_slot + sizeof(float) * B * (n + 16 + gws);
}

pdilqr_status ensure_res(pdilqr_server* sv, Slot& sl, int cls)
{
    ClassRes& r = sl.res[cls];
    if (r.ready) return PDILQR_OK;
    const int nrob = 1 << cls, n = 12 * nrob, nc = 4 * nrob;
    const size_t B = class_cap(sv, cls), S = B * ((size_t)sv->opts.max_N + 1);
    r.n = n;
    r.nc = nc;
    r.slots = (int64_t)S;
    // the largest warp count not above the requested one whose fused kernel
    // fits in shared memory, else one chunk (the sequential sweep, from the
    // global workspace): a chunk of a large state already fills its SM, so
    // more chunks would only add the scan's extra work
    const SizeOps* ops = find_ops(n, n);
    if (!ops || !ops->sqp) return PDILQR_E_INVALID_ARG;
    auto smaller = [](int x) { return x == 16 ? 8 : (x == 8 ? 4 : 1); };
    const bool split = class_split(sv, cls);
    int w = split ? 1 : sv->opts.warps;
    while (w > 1 && (!warps_ok(ops, w) || ops->sqp_smem(w) > kSmemMax || ops->scan_gws_floats(w)))
        w = smaller(w);
    pdilqr_status ps = plan_create_capacity(n, n, (int)B, (int64_t)S, w, &r.plan);
    if (ps != PDILQR_OK) return ps;
    if (split) ps = plan_enable_split(r.plan, kSplitChunks);
    if (ps != PDILQR_OK) {
        pdilqr_plan_destroy(r.plan);
        r.plan = nullptr;
        return ps;
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(dalloc(r, &r.px, S * n)); chk(dalloc(r, &r.pu, S * n)); chk(dalloc(r, &r.pl, S * n));
    chk(dalloc(r, &r.pxr, S * n)); chk(dalloc(r, &r.pur, S * n)); chk(dalloc(r, &r.pct, S * nc));
    chk(dalloc(r, &r.px0, B * n)); chk(dalloc(r, &r.sxr, S * n)); chk(dalloc(r, &r.sur, S * n));
    chk(dalloc(r, &r.sct, S * nc)); chk(dalloc(r, &r.dit, B)); chk(dalloc(r, &r.dst, B));
    chk(dalloc(r, &r.dtab, B));
    chk(halloc(r, &r.htab, B)); chk(halloc(r, &r.hN, B)); chk(halloc(r, &r.horder, B));
    chk(halloc(r, &r.hit, B)); chk(halloc(r, &r.hst, B)); chk(halloc(r, &r.hoff, B));
    chk(halloc(r, &r.hx0, B * n)); chk(halloc(r, &r.hxr, S * n)); chk(halloc(r, &r.hur, S * n));
    chk(halloc(r, &r.hct, S * nc)); chk(halloc(r, &r.hxo, S * n)); chk(halloc(r, &r.huo, S * n));
    if (split) chk(halloc(r, &r.hstage, S));
    if (e != cudaSuccess) {
        free_res(r);
        return e == cudaErrorMemoryAllocation ? PDILQR_E_NO_MEMORY : PDILQR_E_CUDA;
    }
    r.ready = true;
    return PDILQR_OK;
}

void CUDART_CB on_batch_done(void* arg)
{
    // runs on a CUDA callback thread: no CUDA calls here
    auto* pair = static_cast<std::pair<pdilqr_server*, Slot*>*>(arg);
    {
        std::lock_guard<std::mutex> lk(pair->first->mu);
        pair->second->done = true;
    }
    pair->first->cv_work.notify_all();
    delete pair;
}

// Launch one batch on slot `sl` (called without the lock held; the batch's
// requests and clients are owned by the slot until completion).
pdilqr_status launch_batch(pdilqr_server* sv, Slot& sl, std::vector<Request>& reqs,
                           std::vector<Client*>& cls_clients)
{
    const int cls = sl.cls;
    pdilqr_status ps = ensure_res(sv, sl, cls);
    if (ps != PDILQR_OK) return ps;
    ClassRes& r = sl.res[cls];
    const int n = r.n, nc = r.nc, count = (int)reqs.size();
    int64_t off = 0, soff = 0;
    int maxN = 0;
    // longest horizons first in the CTA order
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].N > reqs[b].N; });
    sl.offs.resize(count);
    sl.Ns.resize(count);
    for (int i = 0; i < count; ++i) {
        const Request& q = reqs[i];
        Client& c = *cls_clients[i];
        Entry& e = r.htab[i];
        e.cx = c.x; e.cu = c.u; e.cl = c.l; e.cxr = c.xr; e.cur = c.ur; e.cct = c.ct;
        e.off = off;
        e.N = q.N;
        e.init = (!c.has_state || q.reset) ? 1 : 0;
        e.refs = q.refs ? 1 : 0;
        e.soff = soff;
        e.pad = 0;
        std::memcpy(r.hx0 + (size_t)i * n, q.x0.data(), sizeof(float) * n);
        if (q.refs) {
            std::memcpy(r.hxr + soff * n, q.xr.data(), sizeof(float) * (q.N + 1) * n);
            std::memcpy(r.hur + soff * n, q.ur.data(), sizeof(float) * (q.N + 1) * n);
            std::memcpy(r.hct + soff * nc, q.ct.data(), (size_t)(q.N + 1) * nc);
            soff += q.N + 1;
        }
        r.hN[i] = q.N;
        r.hoff[i] = off;
        sl.offs[i] = off;
        sl.Ns[i] = q.N;
        off += q.N + 1;
        maxN = std::max(maxN, q.N);
    }
    for (int i = 0; i < count; ++i) r.horder[i] = order[i];
    cudaStream_t st = sl.s;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(cudaMemcpyAsync(r.dtab, r.htab, sizeof(Entry) * count, cudaMemcpyHostToDevice, st));
    chk(cudaMemcpyAsync(r.px0, r.hx0, sizeof(float) * count * n, cudaMemcpyHostToDevice, st));
    if (soff) {
        chk(cudaMemcpyAsync(r.sxr, r.hxr, sizeof(float) * soff * n, cudaMemcpyHostToDevice, st));
        chk(cudaMemcpyAsync(r.sur, r.hur, sizeof(float) * soff * n, cudaMemcpyHostToDevice, st));
        chk(cudaMemcpyAsync(r.sct, r.hct, (size_t)soff * nc, cudaMemcpyHostToDevice, st));
    }
    if (e != cudaSuccess) return PDILQR_E_CUDA;
    serve_gather<<<count, 256, 0, st>>>(r.dtab, n, nc, r.sxr, r.sur, r.sct, r.px0, r.px, r.pu, r.pl,
                                        r.pxr, r.pur, r.pct);
    if (cudaGetLastError() != cudaSuccess) return PDILQR_E_CUDA;
    ps = plan_set_batch_async(r.plan, r.hN, r.hoff, r.horder, count, maxN, st);
    if (ps != PDILQR_OK) return ps;
    if (r.hstage) {   // split plan: its linearisation walks the stage map
        for (int64_t k = 0; k < r.slots; ++k) r.hstage[k] = -1;
        for (int i = 0; i < count; ++i)
            for (int k = 0; k <= r.hN[i]; ++k) r.hstage[r.hoff[i] + k] = i;
        ps = plan_set_stage_inst_async(r.plan, r.hstage, st);
        if (ps != PDILQR_OK) return ps;
    }
    pdilqr_srbd_model md = sv->models[cls];
    md.nrob = 1 << cls;
    pdilqr_sqp_opts so{};
    so.max_iters = sv->opts.sqp_iters;
    so.tol_step = 0.f;
    so.tol_theta = 0.f;
    so.c_armijo = 1e-4f;
    so.theta_frac = 1e-2f;
    so.alpha_replay = nullptr;
    pdilqr_sqp_info info{};
    info.iters = r.dit;
    info.status = r.dst;
    ps = pdilqr_solve(r.plan, &md, &so, r.px0, r.px, r.pu, r.pl, r.pxr, r.pur, r.pct, &info,
                      (pdilqr_stream)st);
    if (ps != PDILQR_OK) return ps;
    serve_scatter<<<count, 256, 0, st>>>(r.dtab, n, nc, r.px, r.pu, r.pl, r.pxr, r.pur, r.pct);
    chk(cudaGetLastError());
    chk(cudaMemcpyAsync(r.hxo, r.px, sizeof(float) * off * n, cudaMemcpyDeviceToHost, st));
    chk(cudaMemcpyAsync(r.huo, r.pu, sizeof(float) * off * n, cudaMemcpyDeviceToHost, st));
    chk(cudaMemcpyAsync(r.hit, r.dit, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
    chk(cudaMemcpyAsync(r.hst, r.dst, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
    auto* arg = new (std::nothrow) std::pair<pdilqr_server*, Slot*>(sv, &sl);
    if (!arg) return PDILQR_E_NO_MEMORY;
    chk(cudaLaunchHostFunc(st, on_batch_done, arg));
    if (e != cudaSuccess) return PDILQR_E_CUDA;
    return PDILQR_OK;
}

// With the lock held: record the results of a finished slot.
void complete_slot(pdilqr_server* sv, Slot& sl)
{
    ClassRes& r = sl.res[sl.cls];
    const auto now = Clock::now();
    for (int i = 0; i < sl.count; ++i) {
        auto it = sv->results.find(sl.tickets[i]);
        if (it != sv->results.end()) {
            Result& res = it->second;
            const int n = r.n, N = sl.Ns[i];
            res.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - res.t0).count();
            res.status = r.hst[i];
            res.iters = r.hit[i];
            res.n = n;
            res.N = N;
            res.x.assign(r.hxo + sl.offs[i] * n, r.hxo + (sl.offs[i] + N + 1) * n);
            res.u.assign(r.huo + sl.offs[i] * n, r.huo + (sl.offs[i] + N + 1) * n);
            res.done = true;
            if (sv->lat.size() < kLatRing) sv->lat.push_back(res.latency_ns);
            else sv->lat[sv->lat_pos++ % kLatRing] = res.latency_ns;
        }
        auto c = sv->clients.find(sl.clients[i]);
        if (c != sv->clients.end()) {
            c->second.busy = false;
            c->second.has_state = true;
        }
        sv->completed++;
    }
    sl.busy = false;
    sl.done = false;
    sl.tickets.clear();
    sl.clients.clear();
    sl.count = 0;
    sv->cv_done.notify_all();
}

void worker_loop(pdilqr_server* sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        for (Slot& sl : sv->slots)
            if (sl.busy && sl.done) complete_slot(sv, sl);
        if (sv->stop) {
            bool any = false;
            for (Slot& sl : sv->slots) any = any || sl.busy;
            if (!any) break;
        }
        Slot* free_slot = nullptr;
        for (Slot& sl : sv->slots)
            if (!sl.busy) { free_slot = &sl; break; }
        // the oldest request whose client is idle fixes the size class (a large
        // class only while it leaves a stream for the small ones)
        int large_busy = 0, large_ctas = 0;
        bool split_busy = false;
        for (const Slot& sl : sv->slots) {
            if (sl.busy && sl.cls >= kLargeClass) {
                large_busy += 1;
                large_ctas += sl.count;
            }
            if (sl.busy && class_split(sv, sl.cls)) split_busy = true;
        }
        const int budget = sv->opts.large_cta_budget;
        const bool large_ok = (sv->opts.max_inflight < 2 || large_busy < sv->opts.max_inflight - 1) &&
                              (budget <= 0 || large_ctas < budget);
        int cls = -1;
        for (const Request& q : sv->pending) {
            auto c = sv->clients.find(q.client);
            if (c == sv->clients.end() || c->second.busy) continue;
            const int qc = class_of(q.nrob);
            if (qc >= kLargeClass && !large_ok) continue;
            // one split batch at a time: its cooperative launch needs all of
            // its CTAs resident at once
            if (qc >= 0 && class_split(sv, qc) && split_busy) continue;
            cls = qc;
            break;
        }
        if (!sv->stop && free_slot && cls >= 0) {
            if (sv->opts.batch_window_us > 0 && (int)sv->pending.size() < sv->opts.max_batch) {
                sv->cv_work.wait_for(lk, std::chrono::microseconds(sv->opts.batch_window_us));
            }
            std::vector<Request> reqs;
            std::vector<Client*> cl;
            int cap = class_cap(sv, cls);
            if (cls >= kLargeClass && budget > 0) cap = std::min(cap, budget - large_ctas);
            for (auto it = sv->pending.begin();
                 it != sv->pending.end() && (int)reqs.size() < cap;) {
                auto cit = sv->clients.find(it->client);
                if (cit == sv->clients.end()) { it = sv->pending.erase(it); continue; }
                Client& c = cit->second;
                if (class_of(it->nrob) == cls && !c.busy) {
                    c.busy = true;
                    cl.push_back(&c);
                    reqs.push_back(std::move(*it));
                    it = sv->pending.erase(it);
                } else {
                    ++it;
                }
            }
            Slot& sl = *free_slot;
            sl.busy = true;
            sl.done = false;
            sl.cls = cls;
            sl.count = (int)reqs.size();
            for (const Request& q : reqs) {
                sl.tickets.push_back(q.ticket);
                sl.clients.push_back(q.client);
            }
            sv->batches++;
            sv->batched_requests += sl.count;
            lk.unlock();
            const pdilqr_status ps = launch_batch(sv, sl, reqs, cl);
            lk.lock();
            if (ps != PDILQR_OK) {
                // the batch never reached the GPU: fail its tickets
                for (size_t i = 0; i < reqs.size(); ++i) {
                    auto it = sv->results.find(reqs[i].ticket);
                    if (it != sv->results.end()) {
                        it->second.done = true;
                        it->second.status = ps;
                    }
                    cl[i]->busy = false;
                }
                cudaStreamSynchronize(sl.s);
                sl.busy = false;
                sl.done = false;
                sl.tickets.clear();
                sl.clients.clear();
                sv->cv_done.notify_all();
            }
            continue;
        }
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
}

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" pdilqr_status pdilqr_serve_create(const pdilqr_serve_opts* o, pdilqr_server** out)
{
    if (!out || !o) return PDILQR_E_INVALID_ARG;
    *out = nullptr;
    pdilqr_server* sv = new (std::nothrow) pdilqr_server();
    if (!sv) return PDILQR_E_NO_MEMORY;
    sv->opts = *o;
    for (int c = 0; c < kClasses; ++c) sv->models[c] = o->class_models ? o->class_models[c] : o->model;
    sv->opts.class_models = nullptr;   // read here only
    if (sv->opts.hbm_budget_bytes <= 0) sv->opts.hbm_budget_bytes = int64_t(1) << 30;
    if (sv->opts.hbm_reserve_bytes <= 0) sv->opts.hbm_reserve_bytes = int64_t(256) << 20;
    if (sv->opts.max_batch <= 0) sv->opts.max_batch = 1024;
    if (sv->opts.max_inflight <= 0) sv->opts.max_inflight = 2;
    if (sv->opts.max_N <= 0) sv->opts.max_N = 100;
    if (sv->opts.sqp_iters <= 0) sv->opts.sqp_iters = 1;
    if (sv->opts.warps == 0) sv->opts.warps = 8;
    if (sv->opts.split_max_batch <= 0) sv->opts.split_max_batch = 8;
    const int smr = sv->opts.split_min_robots;
    if (smr != 0 && smr != 4 && smr != 8 && smr != 16) {
        delete sv;
        return PDILQR_E_INVALID_ARG;
    }
    if (sv->opts.max_inflight > 16 || sv->opts.large_cta_budget < 0 || sv->opts.max_N > 4096 ||
        sv->opts.sqp_iters > 32 ||
        (sv->opts.warps != 1 && sv->opts.warps != 4 && sv->opts.warps != 8 && sv->opts.warps != 16)) {
        delete sv;
        return PDILQR_E_INVALID_ARG;
    }
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return PDILQR_E_CUDA;
    }
    if (smr != 0) {
        // a split batch's CTAs must all be resident at once (one SM each at least)
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->device) != cudaSuccess) {
            delete sv;
            return PDILQR_E_CUDA;
        }
        if ((int64_t)sv->opts.split_max_batch * kSplitChunks > sms) {
            delete sv;
            return PDILQR_E_INVALID_ARG;
        }
    }
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)sv->opts.hbm_budget_bytes) != cudaSuccess) {
        delete sv;
        return PDILQR_E_NO_MEMORY;
    }
    sv->pool_base = static_cast<uint8_t*>(p);
    sv->pool.init((size_t)sv->opts.hbm_budget_bytes & ~size_t(255));
    sv->slots.resize(sv->opts.max_inflight);
    for (Slot& sl : sv->slots) {
        if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess) {
            for (Slot& s2 : sv->slots)
                if (s2.s) cudaStreamDestroy(s2.s);
            cudaFree(sv->pool_base);
            delete sv;
            return PDILQR_E_CUDA;
        }
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_serve_submit(pdilqr_server* sv, uint64_t client_id,
                                             const pdilqr_request* q, uint64_t* ticket)
{
    if (!sv || !q || !ticket || !q->x0hat) return PDILQR_E_INVALID_ARG;
    if (class_of(q->nrob) < 0 || q->N < 1 || q->N > sv->opts.max_N)
        return PDILQR_E_INVALID_ARG;
    const bool refs = q->xref != nullptr;
    if (refs && (!q->uref || !q->contact)) return PDILQR_E_INVALID_ARG;
    Request r;
    r.client = client_id;
    r.nrob = q->nrob;
    r.N = q->N;
    r.reset = q->reset;
    r.refs = refs;
    const int n = 12 * q->nrob, S = q->N + 1;
    r.x0.assign(q->x0hat, q->x0hat + n);
    if (refs) {
        r.xr.assign(q->xref, q->xref + (size_t)S * n);
        r.ur.assign(q->uref, q->uref + (size_t)S * n);
        r.ct.assign(q->contact, q->contact + (size_t)S * 4 * q->nrob);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return PDILQR_E_INVALID_ARG;
    auto it = sv->clients.find(client_id);
    if (it == sv->clients.end()) {
        if (!refs) return PDILQR_E_INVALID_ARG;   // a new client brings references
        Client c;
        c.nrob = q->nrob;
        c.n = n;
        c.N = q->N;
        c.bytes = client_bytes(q->nrob, q->N);
        const int cls = class_of(q->nrob);
        if (!sv->class_admitted[cls]) {
            // the class's batch workspace is allocated when its first batch
            // runs: admit its first client only if free memory holds it on
            // every stream that may run the class, plus the reserve
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return PDILQR_E_CUDA;
            const size_t streams = (size_t)(cls >= kLargeClass && sv->opts.max_inflight > 1
                                                ? sv->opts.max_inflight - 1 : sv->opts.max_inflight);
            const size_t need = class_res_bytes(sv, cls) * streams + (size_t)sv->opts.hbm_reserve_bytes;
            if (free_b < need) {
                sv->refused++;
                return PDILQR_E_ADMISSION;
            }
            sv->class_admitted[cls] = true;
        }
        if (!sv->pool.alloc(c.bytes, &c.off)) {
            sv->refused++;
            return PDILQR_E_ADMISSION;
        }
        carve_client(sv, c);
        it = sv->clients.emplace(client_id, c).first;
    } else if (it->second.nrob != q->nrob || it->second.N != q->N) {
        return PDILQR_E_INVALID_ARG;
    }
    r.ticket = sv->next_ticket++;
    r.t0 = Clock::now();
    if (!sv->started) {
        sv->started = true;
        sv->t_first = r.t0;
    }
    Result res0;
    res0.t0 = r.t0;
    sv->results.emplace(r.ticket, res0);
    *ticket = r.ticket;
    sv->pending.push_back(std::move(r));
    sv->submitted++;
    sv->cv_work.notify_all();
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_serve_poll(pdilqr_server* sv, uint64_t ticket, pdilqr_result* res,
                                           int64_t timeout_us)
{
    if (!sv || !res) return PDILQR_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return PDILQR_E_INVALID_ARG;
    const auto deadline = Clock::now() + std::chrono::microseconds(std::max<int64_t>(timeout_us, 0));
    while (!it->second.done) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done)
            return PDILQR_E_TIMEOUT;
        it = sv->results.find(ticket);
        if (it == sv->results.end()) return PDILQR_E_INVALID_ARG;
    }
    Result& r = it->second;
    res->status = r.status;
    res->iters = r.iters;
    res->latency_ns = r.latency_ns;
    if (res->u0 && !r.u.empty()) std::memcpy(res->u0, r.u.data(), sizeof(float) * r.n);
    if (res->x && !r.x.empty()) std::memcpy(res->x, r.x.data(), sizeof(float) * r.x.size());
    if (res->u && !r.u.empty()) std::memcpy(res->u, r.u.data(), sizeof(float) * r.u.size());
    sv->results.erase(it);
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_serve_release(pdilqr_server* sv, uint64_t client_id)
{
    if (!sv) return PDILQR_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->clients.find(client_id);
    if (it == sv->clients.end()) return PDILQR_E_INVALID_ARG;
    if (it->second.busy) return PDILQR_E_INVALID_ARG;
    for (const Request& q : sv->pending)
        if (q.client == client_id) return PDILQR_E_INVALID_ARG;
    sv->pool.release(it->second.off, it->second.bytes);
    sv->clients.erase(it);
    return PDILQR_OK;
}

static pdilqr_status snap_copy(pdilqr_server* sv, uint64_t client_id, float* x, float* u, float* l,
                               const float* xi, const float* ui, const float* li)
{
    if (!sv) return PDILQR_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->clients.find(client_id);
    if (it == sv->clients.end() || it->second.busy) return PDILQR_E_INVALID_ARG;
    Client& c = it->second;
    c.busy = true;   // keep the dispatcher away while copying
    lk.unlock();
    const size_t bytes = sizeof(float) * (size_t)(c.N + 1) * c.n;
    cudaError_t e = cudaSuccess;
    if (x) {
        e = cudaMemcpy(x, c.x, bytes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && u) e = cudaMemcpy(u, c.u, bytes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && l) e = cudaMemcpy(l, c.l, bytes, cudaMemcpyDeviceToHost);
    } else {
        e = cudaMemcpy(c.x, xi, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.u, ui, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.l, li, bytes, cudaMemcpyHostToDevice);
    }
    lk.lock();
    c.busy = false;
    if (!x && e == cudaSuccess) c.has_state = true;
    sv->cv_work.notify_all();
    return e == cudaSuccess ? PDILQR_OK : PDILQR_E_CUDA;
}

extern "C" pdilqr_status pdilqr_serve_snapshot(pdilqr_server* sv, uint64_t client_id, float* x,
                                               float* u, float* lam)
{
    if (!x) return PDILQR_E_INVALID_ARG;
    return snap_copy(sv, client_id, x, u, lam, nullptr, nullptr, nullptr);
}

extern "C" pdilqr_status pdilqr_serve_restore(pdilqr_server* sv, uint64_t client_id,
                                              const float* x, const float* u, const float* lam)
{
    if (!x || !u || !lam) return PDILQR_E_INVALID_ARG;
    return snap_copy(sv, client_id, nullptr, nullptr, nullptr, x, u, lam);
}

extern "C" pdilqr_status pdilqr_serve_stats(pdilqr_server* sv, pdilqr_serve_stats_t* o)
{
    if (!sv || !o) return PDILQR_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    o->submitted = sv->submitted;
    o->completed = sv->completed;
    o->refused = sv->refused;
    o->batches = sv->batches;
    o->clients = (int64_t)sv->clients.size();
    o->pool_bytes_used = (int64_t)sv->pool.used();
    o->pool_bytes_total = (int64_t)sv->pool.total();
    o->mean_batch = sv->batches ? (double)sv->batched_requests / sv->batches : 0.0;
    std::vector<int64_t> v(sv->lat);
    if (!v.empty()) {
        auto q = [&](double f) {
            const size_t k = std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k] / 1e3;
        };
        o->p50_latency_us = q(0.50);
        o->p99_latency_us = q(0.99);
    } else {
        o->p50_latency_us = o->p99_latency_us = 0.0;
    }
    const double secs = sv->started ? std::chrono::duration<double>(Clock::now() - sv->t_first).count() : 0.0;
    o->solves_per_s = secs > 0 ? sv->completed / secs : 0.0;
    return PDILQR_OK;
}

extern "C" pdilqr_status pdilqr_serve_destroy(pdilqr_server* sv)
{
    if (!sv) return PDILQR_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->pending.clear();
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot& sl : sv->slots) {
        if (sl.s) {
            cudaStreamSynchronize(sl.s);
            cudaStreamDestroy(sl.s);
        }
        for (int c = 0; c < kClasses; ++c) free_res(sl.res[c]);
    }
    cudaFree(sv->pool_base);
    delete sv;
    return PDILQR_OK;
}
