// Continuous-batching service (include/lbm_serve.h): many resident D1Q3 /
// D2Q9 simulations in FP32 (1D fixed-state ones in FP64) advanced together by
// one persistent cooperative kernel.
//
// Device side: serve_kernel stays resident and runs round after round.  A
// round walks a work list of tiles of every active simulation -- 1D:
// 256-site strips run by the generic kernel's tile body (step_block); 2D:
// strips of 254 sites x kChunk2 rows run by the strip kernel's body
// (strip_block, any extent) -- with a grid-wide barrier between its K steps.
// Each simulation keeps its own A-B buffers, parity and step budget for the
// round.  Admitted simulations get their start state in their first round;
// a simulation that finishes within a round has its moments computed in the
// same round, after the last step (the tile body with the state update off).
//
// Host side: a service thread admits queued requests first come first
// served while their state fits the device pool, copies their fields and
// each round's work list to the device (copies only, on a second stream),
// and posts the round in a mailbox in mapped host memory; block 0 of the
// kernel polls it (bounded: the kernel leaves after an idle limit and is
// launched again when work arrives) and reports each round done there.
// The loop is pipelined one round deep: round i is posted before the thread
// waits for round i - 1 and copies its finished simulations' moments out, so
// the device never waits for the host's bookkeeping.
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
    StepArgs am;    // moments of the state after the round (fin = 1): write_state 0, mout set
    const double* m;  // init = 1: the start fields (rho, u, T) in device memory
    int init;       // 1: admitted for this round; the round first computes its start state
    int fin;        // 1: the simulation finishes in this round
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

// One tile of simulation S with arguments a (a step, or the moments pass).
// A call, not inlined: inlined into the persistent loop, the tile bodies
// lose registers to values the compiler keeps across rounds and spill; as a
// function each has the whole register budget, for one call per work item.
__device__ __noinline__ void serve_tile(const ServeSim& S, const StepArgs& a, int local, unsigned char* smem) {
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

// The simulation that work item `it` belongs to: the last with item0 <= it.
__device__ __forceinline__ int serve_owner(const ServeSim* sims, int nsims, int it) {
    int lo = 0, hi = nsims - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sims[mid].item0 <= it)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Host <-> kernel mailbox in mapped pinned host memory.  The host posts
// round number `post` after writing its descriptor (and after the round's
// work list and admitted fields have reached device memory); the kernel
// reports `done` after the round's last store.  Rounds are numbered from 1;
// descriptor, timestamps and work list are double-buffered by round parity.
struct RoundDesc {
    int ns, items, K, ninit;
};
struct alignas(64) Mailbox {
    long long post;   // host: last round posted
    long long done;   // kernel: last round completed
    int stop;         // host: 1 = leave at the next poll
    int pad0;
    long long pad[5];
    RoundDesc desc[2];
    unsigned long long t_start[2], t_end[2];  // %globaltimer at round start and end
};
// What block 0 read from the mailbox, for every block (device memory).
struct RoundCtl {
    int status, ns, items, K, ninit;
};

__device__ __forceinline__ long long ld_acquire_sys(const long long* p) {
    long long v;
    asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(long long* p, long long v) {
    asm volatile("st.release.sys.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long serve_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Start state of a simulation admitted for this round (grid-stride over its
// sites and reservoir rows), as init_kernel / reservoir_kernel compute it.
__device__ __noinline__ void serve_init(const ServeSim& S) {
    const StepArgs& a = S.a[0];
    const long long N = a.N, rows = a.rows;
    const double* m = S.m;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, dt = (long long)gridDim.x * blockDim.x;
    const double *rho = m, *u = m + N, *T = m + (1 + S.d) * N;
    for (long long s = t0; s < N; s += dt) {
        if (S.d == 1 && S.dt == DT_F64)
            init_site<1, double>(rho, u, T, static_cast<double*>(S.f[0]), static_cast<double*>(S.b[0]), N, s);
        else if (S.d == 1)
            init_site<1, float>(rho, u, T, static_cast<float*>(S.f[0]), static_cast<float*>(S.b[0]), N, s);
        else
            init_site<2, float>(rho, u, T, static_cast<float*>(S.f[0]), static_cast<float*>(S.b[0]), N, s);
    }
    if (a.fixed_x)
        for (long long t = t0; t < 2 * rows; t += dt) {
            if (S.d == 1 && S.dt == DT_F64)
                reservoir_item<1, double>(rho, u, T, a.nx, rows, N, static_cast<double*>(const_cast<void*>(a.gf)),
                                          static_cast<double*>(const_cast<void*>(a.gb)), static_cast<double*>(const_cast<void*>(a.gaux)), t);
            else if (S.d == 1)
                reservoir_item<1, float>(rho, u, T, a.nx, rows, N, static_cast<float*>(const_cast<void*>(a.gf)),
                                         static_cast<float*>(const_cast<void*>(a.gb)), static_cast<float*>(const_cast<void*>(a.gaux)), t);
            else
                reservoir_item<2, float>(rho, u, T, a.nx, rows, N, static_cast<float*>(const_cast<void*>(a.gf)),
                                         static_cast<float*>(const_cast<void*>(a.gb)), static_cast<float*>(const_cast<void*>(a.gaux)), t);
        }
    if (t0 == 0) *a.flag = 0;
}

// K steps of every simulation in `sims` (sorted by item0), then the moments
// of the simulations that finish in this round.
// The round's parameters (work list parity, simulations, work items, steps)
// are read from shared memory where they are used: kept in registers across
// the round, they would crowd the step bodies (128 registers a thread).
struct RoundShared {
    long long seq;
    int ns, items, K;
};

__device__ __forceinline__ const ServeSim* round_sims(const ServeSim* tables, int max_active,
                                                      const volatile RoundShared* r) {
    return tables + (size_t)(r->seq & 1) * max_active;
}

__device__ __forceinline__ void serve_round(const ServeSim* tables, int max_active,
                                            const volatile RoundShared* r, unsigned char* smem,
                                            cg::grid_group& grid) {
    for (int k = 0; k < r->K; ++k) {
        for (int it = blockIdx.x; it < r->items; it += gridDim.x) {
            const ServeSim* sims = round_sims(tables, max_active, r);
            const ServeSim& S = sims[serve_owner(sims, r->ns, it)];
            if (k >= S.steps) continue;  // uniform over the block
            // read in place (not copied to registers): the tile bodies load
            // the fields they need
            serve_tile(S, S.a[(S.cur + k) & 1], it - S.item0, smem);
        }
        grid.sync();
    }
    // every step of the round is complete (the barrier above): moments
    for (int it = blockIdx.x; it < r->items; it += gridDim.x) {
        const ServeSim* sims = round_sims(tables, max_active, r);
        const ServeSim& S = sims[serve_owner(sims, r->ns, it)];
        if (S.fin) serve_tile(S, S.am, it - S.item0, smem);
    }
}

// The work lists are read with plain (coherent) loads, never through the
// read-only path: the host rewrites a list between the rounds that use it.
//
// The persistent batched kernel: one cooperative launch serves round after
// round.  Block 0 waits for the host to post the next round (bounded: after
// idle_ns without a post, or when the host asks it to stop, every block
// leaves together and the host relaunches when work arrives), then every
// block runs it: start states of the admitted simulations, K steps of every
// active simulation with a grid-wide barrier between steps, moments of the
// finishing ones; block 0 then reports the round done.
__global__ void __launch_bounds__(kTX, 2) serve_kernel(Mailbox* mb, RoundCtl* ctl, const ServeSim* tables,
                                                    int max_active, long long seq0, unsigned long long idle_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ RoundShared rs;
    volatile RoundShared* r = &rs;
    cg::grid_group grid = cg::this_grid();
    volatile RoundCtl* vc = ctl;
    if (threadIdx.x == 0) r->seq = seq0;
    __syncthreads();
    for (;;) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const long long seq = r->seq;
            const int par = (int)(seq & 1);
            int st = 0;
            const unsigned long long t0 = serve_ns();
            unsigned int nap = 128;
            while (ld_acquire_sys(&mb->post) < seq) {
                if (*(volatile int*)&mb->stop) {
                    st = 2;
                    break;
                }
                if (serve_ns() - t0 > idle_ns) {
                    st = 1;
                    break;
                }
                __nanosleep(nap);
                if (nap < 4096) nap *= 2;
            }
            if (st == 0) {
                const volatile RoundDesc* d = &mb->desc[par];
                vc->ns = d->ns;
                vc->items = d->items;
                vc->K = d->K;
                vc->ninit = d->ninit;
                *(volatile unsigned long long*)&mb->t_start[par] = serve_ns();
            }
            vc->status = st;
            __threadfence();
        }
        grid.sync();
        if (vc->status != 0) return;  // every block leaves together
        if (threadIdx.x == 0) {
            r->ns = vc->ns;
            r->items = vc->items;
            r->K = vc->K;
        }
        __syncthreads();
        if (vc->ninit > 0) {
            const ServeSim* sims = round_sims(tables, max_active, r);
            for (int i = 0; i < r->ns; ++i)
                if (sims[i].init) serve_init(sims[i]);
            grid.sync();
        }
        serve_round(tables, max_active, r, smem, grid);
        grid.sync();
        if (threadIdx.x == 0) {
            const long long seq = r->seq;
            if (blockIdx.x == 0) {
                *(volatile unsigned long long*)&mb->t_end[seq & 1] = serve_ns();
                __threadfence_system();
                st_release_sys(&mb->done, seq);
            }
            r->seq = seq + 1;  // every thread of the block has passed its last read (barriers above)
        }
        __syncthreads();
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
    bool fresh = false;  // admitted; its start state is computed by its first round
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
    cudaStream_t stream = nullptr;   // the persistent kernel
    char* pool_mem = nullptr;
    Pool pool;
    cudaStream_t cstream = nullptr;  // copies: admitted fields and work lists in, results out
    ServeSim* d_sims = nullptr;      // [2][max_active]: work lists of rounds i and i + 1
    ServeSim* h_sims = nullptr;      // pinned, [2][max_active]
    int* h_flag = nullptr;           // pinned
    Mailbox* mb = nullptr;           // pinned, mapped: host view
    Mailbox* mb_dev = nullptr;       // device view of the same memory
    RoundCtl* ctl = nullptr;         // device
    bool launched = false;           // a launch of the persistent kernel was made on `stream`
    long long posted = 0;            // rounds posted so far
    uint64_t launches = 0;
    double* stage[2] = {nullptr, nullptr};  // pinned staging of admitted fields, per round parity
    size_t stage_n[2] = {0, 0};             // doubles
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
    bool admit_one(const std::shared_ptr<Request>& r, double* staged);
    bool finish(std::vector<std::shared_ptr<Request>>& done, int par, int nsims);
    bool ensure_kernel();
    bool wait_done(long long seq);
    bool fail_thread(const std::string& m) {
        std::lock_guard<std::mutex> lk(mu);
        thread_error = m;
        cv_done.notify_all();
        return false;
    }
};

long long host_load_acquire(const long long* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
void host_store_release(long long* p, long long v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }

// The persistent kernel runs on `stream` unless it has left (idle limit or
// stop); then it is launched again, starting at the first round not done.
bool Server::ensure_kernel() {
    if (launched) {
        const cudaError_t q = cudaStreamQuery(stream);
        if (q == cudaErrorNotReady) return true;  // still running
        if (q != cudaSuccess) return fail_thread(std::string("serve kernel: ") + cudaGetErrorString(q));
    }
    *(volatile int*)&mb->stop = 0;
    long long seq0 = host_load_acquire(&mb->done) + 1;
    unsigned long long idle_ns = (unsigned long long)(opts.idle_ms * 1e6);
    int ma = opts.max_active;
    void* args[] = {&mb_dev, &ctl, &d_sims, &ma, &seq0, &idle_ns};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)serve_kernel, dim3(grid_max), dim3(kTX), args, kSmem,
                                                stream);
    if (e != cudaSuccess) return fail_thread(std::string("serve kernel launch: ") + cudaGetErrorString(e));
    launched = true;
    ++launches;
    return true;
}

// Wait until round `seq` is done; relaunch the kernel if it left first.
bool Server::wait_done(long long seq) {
    const auto t_start = std::chrono::steady_clock::now();
    unsigned int nap = 2;
    while (host_load_acquire(&mb->done) < seq) {
        if (!ensure_kernel()) return false;
        if (std::chrono::steady_clock::now() - t_start > std::chrono::seconds(600))
            return fail_thread("serve kernel: a round did not complete within 600 s");
        std::this_thread::sleep_for(std::chrono::microseconds(nap));
        if (nap < 200) nap *= 2;
    }
    return true;
}

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

// Device set-up of an admitted request (asynchronous on the server stream):
// its fields, already in pinned staging memory, are copied in and the start
// state (and the reservoirs) computed.
bool Server::admit_one(const std::shared_ptr<Request>& r, double* staged) {
    char* base = pool_mem + r->off;
    double* m = reinterpret_cast<double*>(base + r->lay.m);
    const long long N = r->N;
    // a copy only: no kernel may queue behind the persistent one
    cudaError_t e = cudaMemcpyAsync(m, staged, sizeof(double) * (2 + r->d) * N, cudaMemcpyHostToDevice, cstream);
    if (e != cudaSuccess) return fail_thread(std::string("admission: ") + cudaGetErrorString(e));
    r->cur = 0;
    r->remaining = r->steps;
    r->fresh = true;
    return true;
}

// Round `par` has completed on the device (the caller waited for its end
// event): its time, and the results of the simulations that finished in it
// (moments computed by the round itself) copied to their host vectors.
bool Server::finish(std::vector<std::shared_ptr<Request>>& done, int par, int nsims) {
    const unsigned long long te = *(volatile unsigned long long*)&mb->t_end[par];
    const unsigned long long ts = *(volatile unsigned long long*)&mb->t_start[par];
    const double ms = te > ts ? (te - ts) * 1e-6 : 0.0;
    double done_sites = 0;
    const ServeSim* hs = h_sims + (size_t)par * opts.max_active;
    for (int i = 0; i < nsims; ++i) done_sites += (double)hs[i].a[0].N * hs[i].steps;
    if (ms > 0) rate = 0.5 * rate + 0.5 * done_sites / (ms * 1e-3);
    cudaError_t e = cudaSuccess;
    for (auto& r : done) {
        char* base = pool_mem + r->off;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->fields.data(), base + r->lay.m, sizeof(double) * (2 + r->d) * r->N,
                                cudaMemcpyDeviceToHost, cstream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_flag, base + r->lay.flag, sizeof(int), cudaMemcpyDeviceToHost, cstream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cstream);
        r->flag = *h_flag;
    }
    std::lock_guard<std::mutex> lk(mu);
    busy_s += ms * 1e-3;
    ++rounds;
    if (e != cudaSuccess) {
        thread_error = std::string("results: ") + cudaGetErrorString(e);
        cv_done.notify_all();
        return false;
    }
    n_active -= (int)done.size();
    for (auto& r : done) {
        pool.release(r->off, r->lay.total);
        r->t_done = now_s(t0);
        r->state = 2;
        ++n_completed;
        site_updates += (double)r->N * r->steps;
        last_done = r->t_done;
    }
    if (!done.empty()) cv_done.notify_all();
    return true;
}

void Server::loop() {
    cudaSetDevice(device);
    bool inflight = false;       // round `posted` is on the device
    int inflight_n = 0;          // its number of simulations
    std::vector<std::shared_ptr<Request>> fin[2];  // simulations that finish in the round of that parity
    while (true) {
        std::vector<std::shared_ptr<Request>> admitted;
        bool stopping = false;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active.empty() && !inflight)
                cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop || !queue.empty(); });
            stopping = stop;
            while (!stopping && !queue.empty() && (int)(active.size() + admitted.size()) < opts.max_active) {
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
        if (stopping) {
            // the kernel leaves at its next poll; nothing of the server in
            // flight on return
            *(volatile int*)&mb->stop = 1;
            cudaStreamSynchronize(stream);
            cudaStreamSynchronize(cstream);
            return;
        }
        const long long seq = posted + 1;
        const int par = (int)(seq & 1);
        // admissions: fields into this parity's pinned staging (its last
        // copies, two rounds ago, have completed), then onto the device
        if (!admitted.empty()) {
            size_t need = 0;
            for (auto& r : admitted) need += (size_t)(2 + r->d) * r->N;
            if (need > stage_n[par]) {
                if (stage[par]) cudaFreeHost(stage[par]);
                stage[par] = nullptr;
                stage_n[par] = 0;
                if (cudaMallocHost(&stage[par], sizeof(double) * need) != cudaSuccess) {
                    fail_thread("admission: pinned staging memory");
                    return;
                }
                stage_n[par] = need;
            }
            size_t o = 0;
            for (auto& r : admitted) {
                const size_t n = (size_t)(2 + r->d) * r->N;
                std::memcpy(stage[par] + o, r->fields.data(), sizeof(double) * n);
                if (!admit_one(r, stage[par] + o)) return;
                active.push_back(r);
                o += n;
            }
        }

        // round `seq`: every active simulation advances min(K, remaining)
        // steps; the host's copy of each simulation's step count and parity
        // moves ahead at once (the device follows in round order)
        int ns = (int)active.size();
        fin[par].clear();
        if (ns > 0) {
            double sites = 0;
            long max_rem = 0;
            for (auto& r : active) {
                sites += (double)r->N;
                max_rem = std::max(max_rem, r->remaining);
            }
            long K = (long)(opts.round_ms * 1e-3 * rate / std::max(sites, 1.0));
            K = std::max(1L, std::min({K, max_rem, 4096L}));
            ServeSim* hs = h_sims + (size_t)par * opts.max_active;
            ServeSim* ds = d_sims + (size_t)par * opts.max_active;
            int items = 0, ninit = 0;
            std::vector<std::shared_ptr<Request>> still;
            for (int i = 0; i < ns; ++i) {
                const auto& rp = active[i];
                const Request& r = *rp;
                char* base = pool_mem + r.off;
                ServeSim& sm = hs[i];
                for (int k = 0; k < 2; ++k) {
                    sm.f[k] = base + r.lay.f[k];
                    sm.b[k] = base + r.lay.b[k];
                }
                for (int k = 0; k < 2; ++k) {
                    sm.a[k] = sim_args(*this, r);
                    sm.a[k].fin = sm.f[k];
                    sm.a[k].bin = sm.b[k];
                    sm.a[k].fout = sm.f[k ^ 1];
                    sm.a[k].bout = sm.b[k ^ 1];
                }
                sm.m = reinterpret_cast<const double*>(base + r.lay.m);
                sm.init = r.fresh ? 1 : 0;
                ninit += sm.init;
                rp->fresh = false;
                sm.d = r.d;
                sm.dt = r.dt;
                sm.strip = uses_strip(r) ? 1 : 0;
                sm.tiles_x = sm.strip ? (r.nx + ShS::TX - 1) / ShS::TX : (r.nx + kTX - 1) / kTX;
                sm.item0 = items;
                sm.steps = (int)std::min(K, r.remaining);
                sm.cur = r.cur;
                const int after = r.cur ^ (sm.steps & 1);
                sm.fin = r.remaining - sm.steps <= 0;
                if (sm.fin) {
                    // moments of the final state, as lbm_moments computes them
                    sm.am = sm.a[after];
                    sm.am.write_state = 0;
                    sm.am.mout = reinterpret_cast<double*>(base + r.lay.m);
                }
                items += sm.tiles_x * (r.d == 2 ? (r.ny + kChunk2 - 1) / kChunk2 : 1);
                rp->remaining -= sm.steps;
                rp->cur = after;
                if (sm.fin)
                    fin[par].push_back(rp);
                else
                    still.push_back(rp);
            }
            // the work list and the admitted fields reach device memory
            // before the round is posted
            cudaError_t e = cudaMemcpyAsync(ds, hs, sizeof(ServeSim) * ns, cudaMemcpyHostToDevice, cstream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cstream);
            if (e != cudaSuccess) {
                fail_thread(std::string("round: ") + cudaGetErrorString(e));
                return;
            }
            volatile RoundDesc* d = &mb->desc[par];
            d->ns = ns;
            d->items = items;
            d->K = (int)K;
            d->ninit = ninit;
            host_store_release(&mb->post, seq);
            posted = seq;
            if (!ensure_kernel()) return;
            active.swap(still);
        }

        // round seq - 1: wait for it (round seq is posted behind it), then
        // its results
        if (inflight) {
            if (!wait_done(seq - 1)) return;
            if (!finish(fin[par ^ 1], par ^ 1, inflight_n)) return;
            fin[par ^ 1].clear();
        }
        inflight = ns > 0;
        inflight_n = ns;
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
    o->idle_ms = 50.0;
}

lbm_status lbm_server_create(const lbm_server_opts* opts, lbm_server** out) {
    if (!out) return lbm::serve::fail(LBM_EINVAL, "NULL output handle");
    *out = nullptr;
    lbm_server_opts o;
    lbm_server_default_opts(&o);
    if (opts) o = *opts;
    if (o.max_active <= 0) o.max_active = 4096;
    if (!(o.round_ms > 0)) o.round_ms = 2.0;
    if (!(o.idle_ms > 0)) o.idle_ms = 50.0;
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
        if (S.mb) cudaFreeHost(S.mb);
        if (S.ctl) cudaFree(S.ctl);
        if (S.stream) cudaStreamDestroy(S.stream);
        if (S.cstream) cudaStreamDestroy(S.cstream);
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
        (e = cudaStreamCreateWithFlags(&S.cstream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&S.pool_mem, o.hbm_budget)) != cudaSuccess ||
        (e = cudaMalloc(&S.d_sims, 2 * sizeof(ServeSim) * o.max_active)) != cudaSuccess ||
        (e = cudaMallocHost(&S.h_sims, 2 * sizeof(ServeSim) * o.max_active)) != cudaSuccess ||
        (e = cudaMallocHost(&S.h_flag, sizeof(int))) != cudaSuccess ||
        (e = cudaHostAlloc(&S.mb, sizeof(Mailbox), cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer((void**)&S.mb_dev, S.mb, 0)) != cudaSuccess ||
        (e = cudaMalloc(&S.ctl, sizeof(RoundCtl))) != cudaSuccess)
        return cleanup(std::string("server set-up: ") + cudaGetErrorString(e));
    std::memset(S.mb, 0, sizeof(Mailbox));
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
    o->kernel_launches = S.launches;
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
    // the persistent kernel leaves at its next poll (the worker may have
    // returned on an error without asking it to)
    *(volatile int*)&S.mb->stop = 1;
    cudaStreamSynchronize(S.stream);
    cudaStreamSynchronize(S.cstream);
    cudaFree(S.d_sims);
    cudaFree(S.pool_mem);
    cudaFree(S.ctl);
    cudaFreeHost(S.h_sims);
    cudaFreeHost(S.h_flag);
    cudaFreeHost(S.mb);
    for (int k = 0; k < 2; ++k)
        if (S.stage[k]) cudaFreeHost(S.stage[k]);
    cudaStreamDestroy(S.stream);
    cudaStreamDestroy(S.cstream);
    delete h;
}

}  // extern "C"
