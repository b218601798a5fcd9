// Continuous-batching service (include/lbm_serve.h): many resident D1Q3 /
// D2Q9 simulations in FP32 (1D fixed-state ones in FP64) advanced together by
// one cooperative kernel.
//
// Device side: serve_kernel walks a work list of tiles of every active
// simulation -- 1D: 256-site strips run by the generic kernel's tile body
// (step_block); 2D: strips of 254 sites x kChunk2 rows run by the strip
// kernel's body (strip_block, any extent) -- with a grid-wide
// barrier between steps; it advances the round's K steps in one launch.  Each
// simulation keeps its own A-B buffers, parity and step budget for the round.
//
// Host side: a service thread admits queued requests first come first
// served while their state fits the device pool, launches rounds, and
// retires finished simulations (moments on the device, copy to host).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lbm_serve.h"
#include "lbm_internal.h"
#include "lbm_step_strip.cuh"

namespace lbm {
void set_last_error(const std::string& m);  // lbm_capi.cu
}

namespace lbm {
namespace serve {

namespace cg = cooperative_groups;

constexpr int kTX = 256;     // threads per block, sites per strip
constexpr int kChunk2 = 16;  // rows per 2D work item
constexpr size_t kAlign = 256;

struct ServeSim {
    StepArgs a[2];  // per-simulation arguments for input buffer 0 and 1
    void* f[2];
    void* b[2];
    int d, tiles_x, item0, steps, cur;
    int strip;  // 2D: the strip kernel's body
    int dt;     // storage and arithmetic: DT_F32, or DT_F64 (1D fixed-state requests)
};

using Sh1 = StepShape<1, float, kTX, 1>;
using Sh1d = StepShape<1, double, kTX, 1>;
using ShS = StripShape<float, kTX, true>;  // the serve kernel is register-bound: hand populations over
static_assert(kTX == kStripNT, "the strip body runs on the serve kernel's blocks");
constexpr size_t kmax(size_t x, size_t y) { return x > y ? x : y; }
constexpr size_t kSmem = kmax(kmax(Sh1::smem, Sh1d::smem), (size_t)ShS::SMEM);

// K steps of every simulation in `sims` (sorted by item0); work item `it`
// belongs to the last simulation with item0 <= it.
__global__ void __launch_bounds__(kTX, 2) serve_kernel(const ServeSim* __restrict__ sims, int nsims, int nitems,
                                                    int K) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::grid_group grid = cg::this_grid();
    for (int k = 0; k < K; ++k) {
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            int lo = 0, hi = nsims - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sims[mid].item0 <= it)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const ServeSim& S = sims[lo];
            if (k >= S.steps) continue;  // uniform over the block
            // read in place (not copied to registers): the tile bodies load
            // the fields they need
            const StepArgs& a = S.a[(S.cur + k) & 1];
            const int local = it - S.item0;
            if (S.d == 1) {
                if (S.dt == DT_F64)
                    step_block<1, double, kTX, 1>(a, local, 0, 0, smem);
                else
                    step_block<1, float, kTX, 1>(a, local, 0, 0, smem);
            } else {
                DiagDev<4> acc(0.0f);  // unused: no diagnostics in serving rounds
                int bad = 0;
                if (a.fixed_x)
                    strip_block<float, kTX, true, true>(a, local % S.tiles_x, local / S.tiles_x, smem, acc, bad);
                else
                    strip_block<float, kTX, false, true>(a, local % S.tiles_x, local / S.tiles_x, smem, acc, bad);
                if (bad) atomicOr(a.flag, bad);
            }
            __syncthreads();  // the next work item reuses shared memory
        }
        grid.sync();
    }
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// First-fit allocator over one device allocation (offsets, kAlign granules).
class Pool {
   public:
    size_t size = 0, in_use = 0;
    char* base = nullptr;
    std::map<size_t, size_t> free_;  // offset -> length
    static constexpr size_t npos = ~size_t(0);

    void reset(char* b, size_t n) {
        base = b;
        size = n / kAlign * kAlign;
        free_.clear();
        free_[0] = size;
        in_use = 0;
    }
    size_t alloc(size_t n) {
        n = (n + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            in_use += n;
            return off;
        }
        return npos;
    }
    void release(size_t off, size_t n) {
        n = (n + kAlign - 1) / kAlign * kAlign;
        in_use -= n;
        auto it = free_.emplace(off, n).first;
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
};

// Byte layout of one simulation's device block.
struct Layout {
    size_t f[2], b[2], m, flag, gf, gb, gaux, total;
};

Layout layout_of(int d, long long N, long long rows, bool fixed, int dt) {
    const int Q = d == 1 ? 3 : 9, NB = d == 1 ? 1 : 3;
    const size_t es = dt == DT_F64 ? sizeof(double) : sizeof(float);  // populations, variance, reservoirs
    auto up = [](size_t v) { return (v + kAlign - 1) / kAlign * kAlign; };
    Layout L{};
    size_t o = 0;
    for (int k = 0; k < 2; ++k) {
        L.f[k] = o;
        o += up(es * Q * N);
    }
    for (int k = 0; k < 2; ++k) {
        L.b[k] = o;
        o += up(es * NB * N);
    }
    L.m = o;  // (2 + d) N doubles: initial fields, later the moments
    o += up(sizeof(double) * (2 + d) * N);
    L.flag = o;
    o += kAlign;
    if (fixed) {
        L.gf = o;
        o += up(es * 2 * Q * rows);
        L.gb = o;
        o += up(es * 2 * NB * rows);
        L.gaux = o;
        o += up(es * 2 * (d + NB) * rows);
    }
    L.total = o;
    return L;
}

struct Request {
    uint64_t ticket = 0;
    int d = 1, nx = 1, ny = 1, thermal = 0;
    double tau = 0, T0 = 0;
    lbm_bc bc = LBM_BC_PERIODIC;
    long steps = 0, remaining = 0;
    long long N = 0;
    std::vector<double> fields;  // rho, u (d planes), T; replaced by the result
    double t_submit = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 active, 2 done
    int flag = 0;
    int cur = 0;
    int dt = DT_F32;
    size_t off = 0;
    Layout lay{};
};

// Precision policy: FP32 storage and arithmetic, except 1D fixed-state
// (Riemann) requests, which run in FP64.  In FP32 the 4096-cell two-state
// problem leaves the physical range (rho <= 0) after about 1600 steps --
// rounding-size perturbations at the front grow until they are O(1) -- and
// requests ask for up to 5000 steps; from FP64 rounding the same growth
// takes about three times as many steps, so FP64 carries most of them.  (On
// the longest runs over the longest lattices the scheme leaves the physical
// range in the FP64 oracle too; the server reports those as unstable.)  1D
// lattices are a small share of the work of a mix.
int request_dtype(int d, lbm_bc bc) { return (d == 1 && bc == LBM_BC_FIXED_STATE) ? DT_F64 : DT_F32; }

struct Server {
    lbm_server_opts opts{};
    int device = 0;
    cudaStream_t stream = nullptr;
    char* pool_mem = nullptr;
    Pool pool;
    ServeSim* d_sims = nullptr;
    ServeSim* h_sims = nullptr;  // pinned
    int* h_flag = nullptr;       // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int grid_max = 0;
    std::chrono::steady_clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> active;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::string thread_error;
    std::thread worker;

    // statistics
    uint64_t n_submitted = 0, n_completed = 0;
    int n_active = 0;  // mirrors active.size() for readers holding mu
    double site_updates = 0, busy_s = 0, first_submit = -1, last_done = 0;
    uint64_t rounds = 0;
    double rate = 2e10;  // site updates per second, running estimate for the round length

    void loop();
    bool admit_one(const std::shared_ptr<Request>& r);
    void retire(const std::shared_ptr<Request>& r);
};

// 2D requests run on the strip kernel's tile body.
bool uses_strip(const Request& r) { return r.d == 2; }

StepArgs sim_args(const Server& S, const Request& r) {
    char* base = S.pool_mem + r.off;
    StepArgs a{};
    a.nx = r.nx;
    a.ny = r.ny;
    a.nz = 1;
    a.chunk = r.d == 2 ? kChunk2 : 1;
    a.N = r.N;
    set_step_params(a, r.tau, r.T0);
    a.thermal = r.thermal;
    a.fixed_x = r.bc == LBM_BC_FIXED_STATE;
    a.rows = r.ny;
    if (a.fixed_x) {
        a.gf = base + r.lay.gf;
        a.gb = base + r.lay.gb;
        a.gaux = base + r.lay.gaux;
    }
    a.flag = reinterpret_cast<int*>(base + r.lay.flag);
    a.write_state = 1;
    a.want_diag = 0;
    a.hist_cap = 1;
    return a;
}

// Device set-up of an admitted request (asynchronous on the server stream).
bool Server::admit_one(const std::shared_ptr<Request>& r) {
    char* base = pool_mem + r->off;
    double* m = reinterpret_cast<double*>(base + r->lay.m);
    const long long N = r->N;
    cudaError_t e = cudaMemcpyAsync(m, r->fields.data(), sizeof(double) * (2 + r->d) * N, cudaMemcpyHostToDevice,
                                    stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + r->lay.flag, 0, sizeof(int), stream);
    if (e == cudaSuccess)
        e = launch_init(r->d, r->dt, m, m + N, m + (1 + r->d) * N, base + r->lay.f[0], base + r->lay.b[0], N,
                        stream);
    if (e == cudaSuccess && r->bc == LBM_BC_FIXED_STATE)
        e = launch_reservoir(r->d, r->dt, m, m + N, m + (1 + r->d) * N, r->nx, r->ny, N, base + r->lay.gf,
                             base + r->lay.gb, base + r->lay.gaux, stream);
    if (e != cudaSuccess) {
        thread_error = std::string("admission: ") + cudaGetErrorString(e);
        return false;
    }
    r->cur = 0;
    r->remaining = r->steps;
    return true;
}

// Moments of a finished simulation into its host vector (blocking).
void Server::retire(const std::shared_ptr<Request>& r) {
    char* base = pool_mem + r->off;
    StepArgs a = sim_args(*this, *r);
    a.fin = base + r->lay.f[r->cur];
    a.bin = base + r->lay.b[r->cur];
    a.fout = base + r->lay.f[r->cur ^ 1];
    a.bout = base + r->lay.b[r->cur ^ 1];
    a.write_state = 0;
    a.mout = reinterpret_cast<double*>(base + r->lay.m);
    // the same tile body as the steps (strip kernel, variant 3, for 2D)
    cudaError_t e = launch_step(r->d, r->dt, uses_strip(*r) ? 3 : 0, a, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->fields.data(), a.mout, sizeof(double) * (2 + r->d) * r->N, cudaMemcpyDeviceToHost,
                            stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_flag, a.flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) thread_error = std::string("retire: ") + cudaGetErrorString(e);
    r->flag = *h_flag;
}

void Server::loop() {
    cudaSetDevice(device);
    while (true) {
        std::vector<std::shared_ptr<Request>> admitted;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active.empty())
                cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop || !queue.empty(); });
            if (stop) return;
            while (!queue.empty() && (int)(active.size() + admitted.size()) < opts.max_active) {
                auto r = queue.front();
                const size_t off = pool.alloc(r->lay.total);
                if (off == Pool::npos) break;
                r->off = off;
                r->state = 1;
                queue.pop_front();
                admitted.push_back(r);
                ++n_active;
            }
        }
        for (auto& r : admitted) {
            if (!admit_one(r)) return;
            active.push_back(r);
        }
        if (active.empty()) continue;

        // one round: every active simulation advances min(K, remaining) steps
        double sites = 0;
        long max_rem = 0;
        for (auto& r : active) {
            sites += (double)r->N;
            max_rem = std::max(max_rem, r->remaining);
        }
        long K = (long)(opts.round_ms * 1e-3 * rate / std::max(sites, 1.0));
        K = std::max(1L, std::min({K, max_rem, 4096L}));
        const int ns = (int)active.size();
        int items = 0;
        for (int i = 0; i < ns; ++i) {
            const Request& r = *active[i];
            char* base = pool_mem + r.off;
            ServeSim& s = h_sims[i];
            for (int k = 0; k < 2; ++k) {
                s.f[k] = base + r.lay.f[k];
                s.b[k] = base + r.lay.b[k];
            }
            for (int k = 0; k < 2; ++k) {
                s.a[k] = sim_args(*this, r);
                s.a[k].fin = s.f[k];
                s.a[k].bin = s.b[k];
                s.a[k].fout = s.f[k ^ 1];
                s.a[k].bout = s.b[k ^ 1];
            }
            s.d = r.d;
            s.dt = r.dt;
            s.strip = uses_strip(r) ? 1 : 0;
            s.tiles_x = s.strip ? (r.nx + ShS::TX - 1) / ShS::TX : (r.nx + kTX - 1) / kTX;
            s.item0 = items;
            s.steps = (int)std::min(K, r.remaining);
            s.cur = r.cur;
            items += s.tiles_x * (r.d == 2 ? (r.ny + kChunk2 - 1) / kChunk2 : 1);
        }
        cudaError_t e = cudaMemcpyAsync(d_sims, h_sims, sizeof(ServeSim) * ns, cudaMemcpyHostToDevice, stream);
        int grid = std::max(1, std::min(grid_max, items));
        int Ki = (int)K;
        void* args[] = {&d_sims, (void*)&ns, &items, &Ki};
        if (e == cudaSuccess) e = cudaEventRecord(ev0, stream);
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel((const void*)serve_kernel, dim3(grid), dim3(kTX), args, kSmem, stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            thread_error = std::string("round: ") + cudaGetErrorString(e);
            cv_done.notify_all();
            return;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        double done_sites = 0;
        for (int i = 0; i < ns; ++i) done_sites += (double)active[i]->N * h_sims[i].steps;
        if (ms > 0) rate = 0.5 * rate + 0.5 * done_sites / (ms * 1e-3);

        std::vector<std::shared_ptr<Request>> still;
        std::vector<std::shared_ptr<Request>> finished;
        for (int i = 0; i < ns; ++i) {
            auto& r = active[i];
            r->remaining -= h_sims[i].steps;
            r->cur ^= (h_sims[i].steps & 1);
            if (r->remaining <= 0)
                finished.push_back(r);
            else
                still.push_back(r);
        }
        active.swap(still);
        for (auto& r : finished) retire(r);
        {
            std::lock_guard<std::mutex> lk(mu);
            busy_s += ms * 1e-3;
            ++rounds;
            n_active -= (int)finished.size();
            for (auto& r : finished) {
                pool.release(r->off, r->lay.total);
                r->t_done = now_s(t0);
                r->state = 2;
                ++n_completed;
                site_updates += (double)r->N * r->steps;
                last_done = r->t_done;
            }
            if (!finished.empty()) cv_done.notify_all();
        }
    }
}

lbm_status fail(lbm_status s, const std::string& m) {
    set_last_error(m);
    return s;
}

}  // namespace serve
}  // namespace lbm

using lbm::serve::Server;

struct lbm_server {
    Server s;
};

namespace {

using namespace lbm::serve;

lbm_status copy_out(const Request& r, lbm_fields_out* out, double* latency_s) {
    const long long N = r.N;
    if (out) {
        if (out->rho) std::memcpy(out->rho, r.fields.data(), sizeof(double) * N);
        if (out->u) std::memcpy(out->u, r.fields.data() + N, sizeof(double) * r.d * N);
        if (out->T) std::memcpy(out->T, r.fields.data() + (1 + r.d) * N, sizeof(double) * N);
    }
    if (latency_s) *latency_s = r.t_done - r.t_submit;
    return (r.flag & 1) ? lbm::serve::fail(LBM_EUNSTABLE, "simulation became non-physical (rho <= 0 or not finite)")
                        : LBM_OK;
}

}  // namespace

extern "C" {

void lbm_server_default_opts(lbm_server_opts* o) {
    if (!o) return;
    o->hbm_budget = 0;
    o->max_active = 4096;
    o->device = 0;
    o->round_ms = 2.0;
}

lbm_status lbm_server_create(const lbm_server_opts* opts, lbm_server** out) {
    if (!out) return lbm::serve::fail(LBM_EINVAL, "NULL output handle");
    *out = nullptr;
    lbm_server_opts o;
    lbm_server_default_opts(&o);
    if (opts) o = *opts;
    if (o.max_active <= 0) o.max_active = 4096;
    if (!(o.round_ms > 0)) o.round_ms = 2.0;
    auto* h = new lbm_server();
    Server& S = h->s;
    S.opts = o;
    S.device = o.device;
    S.t0 = std::chrono::steady_clock::now();
    auto cleanup = [&](const std::string& m) {
        if (S.d_sims) cudaFree(S.d_sims);
        if (S.pool_mem) cudaFree(S.pool_mem);
        if (S.h_sims) cudaFreeHost(S.h_sims);
        if (S.h_flag) cudaFreeHost(S.h_flag);
        if (S.ev0) cudaEventDestroy(S.ev0);
        if (S.ev1) cudaEventDestroy(S.ev1);
        if (S.stream) cudaStreamDestroy(S.stream);
        delete h;
        return lbm::serve::fail(LBM_ECUDA, m);
    };
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return cleanup(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cleanup(std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
    if (o.hbm_budget == 0) o.hbm_budget = free_b / 2;
    S.opts.hbm_budget = o.hbm_budget;
    if ((e = cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&S.pool_mem, o.hbm_budget)) != cudaSuccess ||
        (e = cudaMalloc(&S.d_sims, sizeof(ServeSim) * o.max_active)) != cudaSuccess ||
        (e = cudaMallocHost(&S.h_sims, sizeof(ServeSim) * o.max_active)) != cudaSuccess ||
        (e = cudaMallocHost(&S.h_flag, sizeof(int))) != cudaSuccess ||
        (e = cudaEventCreate(&S.ev0)) != cudaSuccess || (e = cudaEventCreate(&S.ev1)) != cudaSuccess)
        return cleanup(std::string("server set-up: ") + cudaGetErrorString(e));
    S.pool.reset(S.pool_mem, o.hbm_budget);
    int per_sm = 0, sms = 0;
    // the strip body needs more than the default 48 KB of dynamic shared memory
    e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, kTX, kSmem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device);
    if (e != cudaSuccess || per_sm < 1) return cleanup("serve kernel occupancy query failed");
    S.grid_max = per_sm * sms;
    S.worker = std::thread([&S] { S.loop(); });
    *out = h;
    return LBM_OK;
}

lbm_status lbm_server_submit(lbm_server* h, const lbm_request* q, uint64_t* ticket) {
    if (!h || !q || !ticket) return lbm::serve::fail(LBM_EINVAL, "NULL argument");
    if (q->dim < 1 || q->dim > 2) return lbm::serve::fail(LBM_EINVAL, "dim must be 1 or 2");
    if (q->nx < 2 || q->ny < 1 || (q->dim == 1 && q->ny != 1) || (q->dim == 2 && q->ny < 2))
        return lbm::serve::fail(LBM_EINVAL, "invalid extents");
    if (!(q->tau > 0) || !(q->T0 > 0) || q->steps < 0) return lbm::serve::fail(LBM_EINVAL, "invalid tau, T0 or steps");
    if (q->bc != LBM_BC_PERIODIC && q->bc != LBM_BC_FIXED_STATE) return lbm::serve::fail(LBM_EINVAL, "invalid bc");
    if (!q->rho || !q->u || !q->T) return lbm::serve::fail(LBM_EINVAL, "NULL field");
    Server& S = h->s;
    auto r = std::make_shared<Request>();
    r->d = q->dim;
    r->nx = q->nx;
    r->ny = q->ny;
    r->tau = q->tau;
    r->T0 = q->T0;
    r->thermal = q->thermal ? 1 : 0;
    r->bc = q->bc;
    r->steps = q->steps;
    r->N = (long long)q->nx * q->ny;
    r->dt = request_dtype(r->d, r->bc);
    r->lay = layout_of(r->d, r->N, r->ny, r->bc == LBM_BC_FIXED_STATE, r->dt);
    if (r->lay.total > S.pool.size) return lbm::serve::fail(LBM_ENOMEM, "request larger than the server's pool");
    const long long N = r->N;
    r->fields.resize((size_t)(2 + r->d) * N);
    std::memcpy(r->fields.data(), q->rho, sizeof(double) * N);
    std::memcpy(r->fields.data() + N, q->u, sizeof(double) * r->d * N);
    std::memcpy(r->fields.data() + (1 + r->d) * N, q->T, sizeof(double) * N);
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (!S.thread_error.empty()) return lbm::serve::fail(LBM_ECUDA, S.thread_error);
        r->ticket = S.next_ticket++;
        r->t_submit = now_s(S.t0);
        if (S.first_submit < 0) S.first_submit = r->t_submit;
        ++S.n_submitted;
        S.tickets[r->ticket] = r;
        S.queue.push_back(r);
        *ticket = r->ticket;
    }
    S.cv_work.notify_one();
    return LBM_OK;
}

lbm_status lbm_server_wait(lbm_server* h, uint64_t ticket, double timeout_s, lbm_fields_out* out,
                           double* latency_s) {
    if (!h) return lbm::serve::fail(LBM_EINVAL, "NULL server");
    Server& S = h->s;
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(S.mu);
        auto it = S.tickets.find(ticket);
        if (it == S.tickets.end()) return lbm::serve::fail(LBM_EINVAL, "unknown ticket");
        r = it->second;
        const auto until = std::chrono::steady_clock::now() +
                           std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                               std::chrono::duration<double>(std::max(timeout_s, 0.0)));
        S.cv_done.wait_until(lk, until, [&] { return r->state == 2 || !S.thread_error.empty(); });
        if (!S.thread_error.empty()) return lbm::serve::fail(LBM_ECUDA, S.thread_error);
        if (r->state != 2) return lbm::serve::fail(LBM_EBUSY, "request not finished");
        S.tickets.erase(ticket);
    }
    return copy_out(*r, out, latency_s);
}

lbm_status lbm_server_poll(lbm_server* h, uint64_t ticket, lbm_fields_out* out, double* latency_s) {
    return lbm_server_wait(h, ticket, 0.0, out, latency_s);
}

lbm_status lbm_server_stats_get(lbm_server* h, lbm_server_stats* o) {
    if (!h || !o) return lbm::serve::fail(LBM_EINVAL, "NULL argument");
    Server& S = h->s;
    std::lock_guard<std::mutex> lk(S.mu);
    o->submitted = S.n_submitted;
    o->completed = S.n_completed;
    o->active = S.n_active;
    o->queued = (int)S.queue.size();
    o->site_updates = S.site_updates;
    o->busy_s = S.busy_s;
    o->rounds = S.rounds;
    o->first_submit_s = S.first_submit;
    o->last_done_s = S.last_done;
    o->pool_bytes = S.pool.size;
    o->pool_in_use = S.pool.in_use;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* h) {
    if (!h) return;
    Server& S = h->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
    }
    S.cv_work.notify_all();
    if (S.worker.joinable()) S.worker.join();
    cudaStreamSynchronize(S.stream);
    cudaFree(S.d_sims);
    cudaFree(S.pool_mem);
    cudaFreeHost(S.h_sims);
    cudaFreeHost(S.h_flag);
    cudaEventDestroy(S.ev0);
    cudaEventDestroy(S.ev1);
    cudaStreamDestroy(S.stream);
    delete h;
}

}  // extern "C"
