// C-ABI runtime of the bump-function lattice Boltzmann library: simulation
// objects, device buffers (A-B ping-pong of the emitted state), the tile /
// chunk autotuner, CUDA-graph replay of step sequences, moments,
// diagnostics and checkpoints.  See include/lbm.h for the contract.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

int q_of(int D) { return D == 3 ? 19 : (D == 2 ? 9 : 3); }
int nb_of(int D) { return D == 3 ? 6 : (D == 2 ? 3 : 1); }
size_t fbytes_of(int dtype) { return dtype == DT_F64 ? 8 : (dtype == DT_F32 ? 4 : 2); }
size_t rbytes_of(int dtype) { return dtype == DT_F64 ? 8 : 4; }

// autotune cache: (D, dtype, nx, ny, nz) -> (variant, chunk)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::pair<int, int>> g_tune;

const int kHistCap = 4096;

}  // namespace

namespace lbm {
// Error message of the calling thread for lbm_last_error(), set by entry
// points implemented in other translation units.
void set_last_error(const std::string& m) { g_err = m; }
}  // namespace lbm

struct lbm_sim {
    int D = 0, Q = 0, NB = 0;
    int nx = 1, ny = 1, nz = 1;
    long long N = 0, rows = 0;
    double tau = 0, T0 = 0;
    int bc = 0;
    double acc[3] = {0, 0, 0};  // body-force acceleration
    bool forced = false;
    double uw[2][3] = {{0, 0, 0}, {0, 0, 0}};  // wall velocities (lower, upper)
    bool walls_moving = false;
    bool mrt = false;  // MRT collision (D3Q19) with rates mrt_s
    int debug = 0;     // LBM_DEBUG_* flags (lbm_set_debug)
    double small_t = 0;  // lbm_set_small_t: FP64 temperature recovery where T < small_t |u|^2
    void* aux = nullptr;  // opts.inplace: (u0, rho b) planes between the two passes
    double mrt_s[2] = {0, 0};
    lbm_opts opts{};
    int dtype = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* f[2] = {nullptr, nullptr};
    void* b[2] = {nullptr, nullptr};
    int cur = 0;
    void* gf = nullptr;
    void* gb = nullptr;
    void* gaux = nullptr;
    double* partial = nullptr;
    size_t partial_blocks = 0;
    unsigned int* ticket = nullptr;
    double* hist = nullptr;
    long long* step_ctr = nullptr;
    int* flag = nullptr;
    double* diag_out = nullptr;
    double* fields = nullptr;  // (D+2) N doubles: init input / moments output
    int var = -1, chunk = 0;
    int multi_k = 0;  // steps per multi-step launch (0: not decided, 1: single steps)
    int cluster_v = -1;  // >= 0: the multi-step launches run the cluster-resident kernel, variant cluster_v
    long nstep = 0;
    // graphs: [parity of cur] -> executable graph of kGraphSteps launches
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_steps = 0;
    // tensor maps of the TMA-staged kernel: variant -> per input buffer (f, b)
    std::map<int, std::array<std::pair<CUtensorMap, CUtensorMap>, 2>> tmaps;
    std::vector<std::pair<void*, size_t>> allocs;

    void* dalloc(size_t bytes) {
        void* p = nullptr;
        if (bytes == 0) bytes = 16;
        if (opts.alloc) {
            p = opts.alloc(bytes, opts.alloc_ctx);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) allocs.push_back({p, bytes});
        return p;
    }
    void release() {
        for (int k = 0; k < 2; ++k)
            if (graph[k]) cudaGraphExecDestroy(graph[k]);
        for (auto& a : allocs) {
            if (opts.alloc && opts.free)
                opts.free(a.first, a.second, opts.alloc_ctx);
            else if (!opts.alloc)
                cudaFree(a.first);
        }
        allocs.clear();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

StepArgs base_args(const lbm_sim* s) {
    StepArgs a{};
    a.fin = s->f[s->cur];
    a.bin = s->b[s->cur];
    a.fout = s->f[1 - s->cur];
    a.bout = s->b[1 - s->cur];
    a.nx = s->nx;
    a.ny = s->ny;
    a.nz = s->nz;
    a.chunk = s->chunk;
    a.halo = s->opts.halo;
    a.N = s->N;
    set_step_params(a, s->tau, s->T0);
    a.thermal = s->opts.thermal;
    a.fixed_x = s->bc == LBM_BC_FIXED_STATE;
    a.walls = s->bc == LBM_BC_WALLS;
    a.forced = s->forced ? 1 : 0;
    for (int c = 0; c < 3; ++c) {
        a.acc[c] = s->acc[c];
        a.acc_f[c] = (float)s->acc[c];
    }
    a.walls_moving = s->walls_moving ? 1 : 0;
    a.mrt = s->mrt ? 1 : 0;
    a.debug_missing_copy = (s->debug & LBM_DEBUG_MISSING_COPY) ? 1 : 0;
    a.small_t = s->small_t;
    a.small_t_f = (float)s->small_t;
    for (int k = 0; k < 2; ++k) {
        a.mrt_s[k] = s->mrt_s[k];
        a.mrt_s_f[k] = (float)s->mrt_s[k];
    }
    for (int w = 0; w < 2; ++w)
        for (int c = 0; c < 3; ++c) {
            a.uw[w][c] = s->uw[w][c];
            a.uw_f[w][c] = (float)s->uw[w][c];
        }
    a.rows = s->rows;
    a.gf = s->gf;
    a.gb = s->gb;
    a.gaux = s->gaux;
    a.partial = s->partial;
    a.ticket = s->ticket;
    a.step_ctr = s->step_ctr;
    a.flag = s->flag;
    a.hist_cap = kHistCap;
    return a;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Walls, the body force, the MRT collision and the FP64 small-T recovery are
// implemented in the generic kernel only: the
// staged, strip and serving kernels serve periodic and fixed-state lattices.
bool small_t_on(const lbm_sim* s) { return s->small_t > 0 && s->opts.thermal && s->dtype != DT_F64; }
bool generic_only(const lbm_sim* s) { return s->bc == LBM_BC_WALLS || s->forced || s->mrt || small_t_on(s); }
// The staged kernel's force/MRT tile serves forced or MRT lattices that are
// periodic, FP32 and without the small-T recovery.
bool ext_ok(const lbm_sim* s) {
    return (s->forced || s->mrt) && s->bc == LBM_BC_PERIODIC && s->dtype == DT_F32 && s->D >= 2 && !small_t_on(s) &&
           s->opts.model == LBM_MODEL_BUMP && !s->opts.inplace;
}
// The staged kernel's walls tile serves walled FP32 lattices (with or
// without force and MRT) without the small-T recovery.
bool walls_ok(const lbm_sim* s) {
    return s->bc == LBM_BC_WALLS && s->dtype == DT_F32 && s->D >= 2 && !small_t_on(s) &&
           s->opts.model == LBM_MODEL_BUMP && !s->opts.inplace && s->opts.halo == 0;
}
// 0: not one of the staged kernel's own tiles; 1: force/MRT tile; 2: walls tile
int own_kind_of(const lbm_sim* s, int v) {
    return (v >= kOwnBase && v < kOwnBase + n_own_variants(s->D)) ? own_kind(s->D, v - kOwnBase) : 0;
}
bool variant_allowed(const lbm_sim* s, int v) {
    const int kind = own_kind_of(s, v);
    if (kind == 1) return ext_ok(s);
    if (kind == 2) return walls_ok(s);
    if (!generic_only(s)) return true;
    return v < kTmaBase && !(s->D == 2 && v == 3);
}

// The TMA-staged kernel needs FP32/16-bit storage, tiles that divide the
// extents, and rows whose byte length is a multiple of 16 (tensor strides).
bool tma_applicable(const lbm_sim* s, int v) {
    if (v < kTmaBase || s->D < 2 || s->dtype == DT_F64) return false;
    if (v >= kOwnBase && v < kPairBase) {
        // FP32-only tiles: the force/MRT tile for forced or MRT periodic
        // lattices, the walls tile for walled ones
        const int kind = own_kind_of(s, v);
        if (kind == 0 || (kind == 1 && !ext_ok(s)) || (kind == 2 && !walls_ok(s))) return false;
    } else if (generic_only(s)) {
        return false;
    } else if (v >= kPairBase) {
        // the pair kernel: periodic lattices; FP32 storage, and in 2D also
        // 16-bit storage
        if (v - kPairBase >= n_pair_variants(s->D)) return false;
        if ((s->dtype != DT_F32 && s->D != 2) || s->bc != LBM_BC_PERIODIC) return false;
    } else if (v - kTmaBase >= n_tma_variants(s->D)) {
        return false;
    }
    Variant t = variant(s->D, v);
    if (s->nx % t.tx != 0) return false;
    if (s->D == 3 && s->ny % t.ty != 0) return false;
    if ((s->nx * fbytes_of(s->dtype)) % 16 != 0 || (s->nx * 4) % 16 != 0) return false;
    if (s->nx < 2 || (s->D == 3 && s->ny < 2)) return false;
    // the march index wraps with one conditional add or subtract
    if ((s->D == 3 ? s->nz : s->ny) < 4) return false;
    // plane offsets i N + s and variance offsets are 32-bit in the staged kernels
    if ((long long)s->Q * s->N >= (1LL << 31)) return false;
    return encode_fn() != nullptr;
}

lbm_status tma_maps(lbm_sim* s, int v, int buf, TmaArgs* ta) {
    auto it = s->tmaps.find(v);
    if (it == s->tmaps.end()) {
        TmaBox box{};
        CK(tma_box(s->D, s->dtype, v, &box));
        std::array<std::pair<CUtensorMap, CUtensorMap>, 2> maps{};
        auto enc = encode_fn();
        const cuuint64_t es = fbytes_of(s->dtype);
        const CUtensorMapDataType dt = s->dtype == DT_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                       : s->dtype == DT_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        const cuuint64_t nx = s->nx, ny = s->ny, nz = s->nz, N = s->N;
        for (int k = 0; k < 2; ++k) {
            cuuint32_t estr[4] = {1, 1, 1, 1};
            CUresult r1, r2;
            if (s->D == 3) {
                cuuint64_t gd[4] = {nx, ny, nz, (cuuint64_t)s->Q};
                cuuint64_t gs[3] = {nx * es, nx * ny * es, N * es};
                cuuint32_t bx[4] = {(cuuint32_t)box.sxf, (cuuint32_t)box.sy, 1, (cuuint32_t)s->Q};
                r1 = enc(&maps[k].first, dt, 4, s->f[k], gd, gs, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                // variance: three planes of component pairs, (2 nx) floats per row
                cuuint64_t gdb[4] = {2 * nx, ny, nz, (cuuint64_t)s->NB / 2};
                cuuint64_t gsb[3] = {2 * nx * 4, 2 * nx * ny * 4, 2 * N * 4};
                cuuint32_t bxb[4] = {2 * (cuuint32_t)box.sxb, (cuuint32_t)box.sy, 1, (cuuint32_t)s->NB / 2};
                r2 = enc(&maps[k].second, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, s->b[k], gdb, gsb, bxb, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            } else {
                cuuint64_t gd[3] = {nx, ny, (cuuint64_t)s->Q};
                cuuint64_t gs[2] = {nx * es, N * es};
                cuuint32_t bx[3] = {(cuuint32_t)box.sxf, 1, (cuuint32_t)s->Q};
                r1 = enc(&maps[k].first, dt, 3, s->f[k], gd, gs, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                cuuint64_t gdb[3] = {nx, ny, (cuuint64_t)s->NB};
                cuuint64_t gsb[2] = {nx * 4, N * 4};
                cuuint32_t bxb[3] = {(cuuint32_t)box.sxb, 1, (cuuint32_t)s->NB};
                r2 = enc(&maps[k].second, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, s->b[k], gdb, gsb, bxb, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            }
            if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
                return fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r1) + ", " +
                                           std::to_string((int)r2) + ")");
        }
        it = s->tmaps.emplace(v, maps).first;
    }
    ta->fmap = it->second[buf].first;
    ta->bmap = it->second[buf].second;
    return LBM_OK;
}

// Launch variant v with arguments a; `buf` is the input buffer (a.fin).
lbm_status launch_variant(lbm_sim* s, int v, const StepArgs& a, int buf) {
    if (v == kInplaceVariant) {
        // the memory form of the population buffer is the parity of the state
        CK(launch_step_aa(s->D, s->dtype, a, buf, s->aux, s->stream));
    } else if (v == kStdVariant) {
        CK(launch_std_step(s->D, s->dtype, a, s->stream));
    } else if (v >= kTmaBase) {
        TmaArgs ta;
        lbm_status st = tma_maps(s, v, buf, &ta);
        if (st != LBM_OK) return st;
        ta.s = a;
        CK(launch_step_tma(s->D, s->dtype, v, ta, s->stream));
    } else {
        CK(launch_step(s->D, s->dtype, v, a, s->stream));
    }
    return LBM_OK;
}

size_t blocks_of(const lbm_sim* s, int v, int chunk) {
    if (v == kInplaceVariant) return (size_t)((s->N + 255) / 256);
    dim3 g = step_grid(s->D, v, s->nx, s->ny, s->nz, chunk);
    return (size_t)g.x * g.y * g.z;
}

// Chunk candidates along the march axis: keep at least ~4 waves of blocks on
// 152 SMs while amortising the two-plane ring of each chunk.
std::vector<int> chunk_candidates(const lbm_sim* s) {
    int np = (s->D == 3 ? s->nz : (s->D == 2 ? s->ny : 1)) - (s->D >= 2 ? 2 * s->opts.halo : 0);
    if (s->D == 1) return {1};
    std::vector<int> c;
    // lattices of few planes: short marches (more blocks, less latency per step)
    if (np <= 1024) {
        c.push_back(2);
        c.push_back(4);
    }
    for (int k : {8, 10, 12, 14, 16, 20, 24, 28, 32, 64, 128, 256}) {
        if (k >= np) {
            c.push_back(np);
            break;
        }
        c.push_back(k);
    }
    return c;
}

lbm_status ensure_partial(lbm_sim* s, int v, int chunk) {
    size_t nb = blocks_of(s, v, chunk);
    if (nb <= s->partial_blocks) return LBM_OK;
    double* p = (double*)s->dalloc(nb * (s->D + 2) * sizeof(double));
    if (!p) return fail(LBM_ENOMEM, "diagnostics partial buffer");
    s->partial = p;
    s->partial_blocks = nb;
    return LBM_OK;
}

lbm_status launch_one_step(lbm_sim* s, bool diag) {
    StepArgs a = base_args(s);
    a.write_state = 1;
    a.want_diag = diag ? 1 : 0;
    a.hist = s->hist;
    lbm_status st = launch_variant(s, s->var, a, s->cur);
    if (st != LBM_OK) return st;
    s->cur = 1 - s->cur;
    return LBM_OK;
}

// K steps of a D1 or small D2 lattice in one cooperative launch from the
// current buffer.
lbm_status launch_multi(lbm_sim* s, int K, bool diag, void* const* f, void* const* b) {
    StepArgs a[2];
    for (int p = 0; p < 2; ++p) {
        a[p] = base_args(s);
        a[p].fin = f[p];
        a[p].bin = b[p];
        a[p].fout = f[1 - p];
        a[p].bout = b[1 - p];
        a[p].write_state = 1;
        a[p].want_diag = diag ? 1 : 0;
        a[p].hist = s->hist;
    }
    const int c = s->cur;
    cudaError_t e;
    if (s->D == 2 && s->cluster_v >= 0) {
        e = launch_step_cluster_d2(s->dtype, s->cluster_v, a[c], a[1 - c], K, s->stream);
    } else if (s->D == 2) {
        for (int p = 0; p < 2; ++p) a[p].chunk = kMultiChunk2;
        e = launch_step_multi_d2(s->dtype, a[c], a[1 - c], K, s->stream);
    } else {
        e = launch_step_multi_d1(s->dtype, s->var, a[c], a[1 - c], K, s->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, std::string("multi-step launch: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

// Steps per launch (D1, and D2 lattices of at most kMulti2Sites sites, where a
// step takes about as long as a launch).  opts.steps_per_launch > 1 forces a
// length; 0 times a replay of 64 single-step launches (CUDA graph) against
// one 64-step cooperative launch and, for periodic D2 lattices that fit the
// shared memory of a thread-block cluster, against 64 steps of each cluster
// variant, on scratch copies of the state, and keeps the fastest.
constexpr long long kMulti2Sites = 1LL << 18;

// The cluster-resident kernel serves periodic D2 bump lattices in FP32/FP64
// without the generic kernel's settings (walls, force, MRT, small-T).
bool cluster_applicable(const lbm_sim* s, int v) {
    return s->D == 2 && s->bc == LBM_BC_PERIODIC && s->opts.model != LBM_MODEL_STANDARD && !s->opts.inplace &&
           !s->opts.halo && !generic_only(s) && (s->dtype == DT_F32 || s->dtype == DT_F64) &&
           cluster_fits_d2(s->dtype, v, s->nx, s->ny) &&
           launch_step_cluster_d2(s->dtype, v, base_args(s), base_args(s), 1, s->stream, true) == cudaSuccess;
}

// Shortest of three timed runs of `run` (CUDA events on stream st); 1e30 if
// the events fail.
template <typename F> float best_of(cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st, F run) {
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        float t = 1e30f;
        cudaEventRecord(e0, st);
        run();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t < best)
            best = t;
    }
    return best;
}

lbm_status tune_multi(lbm_sim* s) {
    s->multi_k = 1;
    s->cluster_v = -1;
    cudaGetLastError();
    // forced cluster variant (opts.cluster = 1 + v); a setting only the
    // generic kernel has (force, MRT, small-T) takes precedence
    if (s->opts.cluster > 0 && !generic_only(s)) {
        const int v = s->opts.cluster - 1;
        if (!cluster_applicable(s, v)) {
            cudaGetLastError();
            return fail(LBM_EINVAL, "opts.cluster: the lattice does not fit that cluster variant "
                                    "(periodic D2 bump lattice, FP32/FP64, no halo, rows >= blocks, "
                                    "state within the cluster's shared memory)");
        }
        if ((size_t)cluster_blocks(v) > s->partial_blocks) {
            double* p = (double*)s->dalloc((size_t)cluster_blocks(v) * (s->D + 2) * sizeof(double));
            if (!p) return fail(LBM_ENOMEM, "diagnostics partial buffer");
            s->partial = p;
            s->partial_blocks = cluster_blocks(v);
        }
        s->cluster_v = v;
        s->multi_k = s->opts.steps_per_launch > 1 ? s->opts.steps_per_launch : 64;
        return LBM_OK;
    }
    // D2: only for autotuned tiles (a forced tile runs as asked) or when the
    // caller asks for a length
    const bool small2 = s->D == 2 && s->N <= kMulti2Sites && !s->opts.halo &&
                        (s->opts.tile < 0 || s->opts.steps_per_launch > 1);
    if ((s->D != 1 && !small2) || s->opts.steps_per_launch == 1 || s->opts.model == LBM_MODEL_STANDARD ||
        s->opts.inplace)
        return LBM_OK;
    if (s->D == 2) {
        // the cooperative D2 launch has a fixed tiling: diagnostics partials for it
        const size_t nb = (size_t)((s->nx + kMultiTX2 - 1) / kMultiTX2) * ((s->ny + kMultiChunk2 - 1) / kMultiChunk2);
        if (nb > s->partial_blocks) {
            double* p = (double*)s->dalloc(nb * (s->D + 2) * sizeof(double));
            if (!p) return fail(LBM_ENOMEM, "diagnostics partial buffer");
            s->partial = p;
            s->partial_blocks = nb;
        }
    }
    if (s->opts.steps_per_launch > 1) {  // forced
        s->multi_k = s->opts.steps_per_launch;
        return LBM_OK;
    }
    const int K = 64;
    // scratch copies of the state, from the caller's allocator if one is set
    auto tmp_alloc = [s](size_t n) -> void* {
        void* p = nullptr;
        if (s->opts.alloc) return s->opts.alloc(n, s->opts.alloc_ctx);
        return cudaMalloc(&p, n) == cudaSuccess ? p : nullptr;
    };
    auto tmp_free = [s](void* p, size_t n) {
        if (!p) return;
        if (s->opts.alloc)
            s->opts.free(p, n, s->opts.alloc_ctx);
        else
            cudaFree(p);
    };
    const size_t fb = (size_t)s->Q * s->N * fbytes_of(s->dtype), bb = (size_t)s->NB * s->N * rbytes_of(s->dtype);
    void *tf[2] = {nullptr, nullptr}, *tb[2] = {nullptr, nullptr};
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        tf[k] = tmp_alloc(fb);
        tb[k] = tmp_alloc(bb);
        ok = tf[k] && tb[k];
    }
    float t_multi = 1e30f, t_graph = 1e30f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the scratch runs may raise the flag word on a bad state: keep its value
    int flag0 = 0;
    if (cudaMemcpy(&flag0, s->flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
    if (ok) ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (ok) {
        for (int k = 0; k < 2; ++k) {
            cudaMemcpyAsync(tf[k], s->f[s->cur], fb, cudaMemcpyDeviceToDevice, s->stream);
            cudaMemcpyAsync(tb[k], s->b[s->cur], bb, cudaMemcpyDeviceToDevice, s->stream);
        }
        // the timing runs write a scratch flag word only if the state is bad;
        // diagnostics off, the history untouched
        if (launch_multi(s, K, false, tf, tb) == LBM_OK)
            t_multi = best_of(e0, e1, s->stream, [&] { launch_multi(s, K, false, tf, tb); });
        cudaGetLastError();
        {
            // single steps on the same scratch buffers, captured as one graph
            void* sf[2] = {s->f[0], s->f[1]};
            void* sb[2] = {s->b[0], s->b[1]};
            // the staged kernels' tensor maps are cached per variant with the
            // buffers they were built for: keep the real buffers' maps aside,
            // and drop every map built for the scratch buffers afterwards
            auto saved_maps = s->tmaps;
            s->tmaps.clear();
            s->f[0] = tf[0], s->f[1] = tf[1], s->b[0] = tb[0], s->b[1] = tb[1];
            cudaGraphExec_t ge = nullptr;
            cudaGraph_t g;
            if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                lbm_status st = LBM_OK;
                for (int k = 0; k < K && st == LBM_OK; ++k) st = launch_one_step(s, false);
                if (cudaStreamEndCapture(s->stream, &g) == cudaSuccess) {
                    if (st == LBM_OK && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
                        cudaGraphLaunch(ge, s->stream);
                        t_graph = best_of(e0, e1, s->stream, [&] { cudaGraphLaunch(ge, s->stream); });
                        cudaGraphExecDestroy(ge);
                    }
                    cudaGraphDestroy(g);
                }
            }
            cudaGetLastError();
            s->f[0] = sf[0], s->f[1] = sf[1], s->b[0] = sb[0], s->b[1] = sb[1];
            cudaStreamSynchronize(s->stream);  // the scratch runs are done before their maps go
            s->tmaps = saved_maps;
            // launch_one_step flipped s->cur K times: K is even
        }
    }
    // the cluster-resident kernel (periodic D2 lattices that fit), each variant
    float t_cluster = 1e30f;
    int best_cluster = -1;
    if (ok && s->D == 2 && s->opts.cluster == 0) {
        for (int v = 0; v < n_cluster_variants(); ++v) {
            if (!cluster_applicable(s, v)) {
                cudaGetLastError();
                continue;
            }
            s->cluster_v = v;
            float t = 1e30f;
            if (launch_multi(s, K, false, tf, tb) == LBM_OK)
                t = best_of(e0, e1, s->stream, [&] { launch_multi(s, K, false, tf, tb); });
            cudaGetLastError();
            s->cluster_v = -1;
            if (t < t_cluster) {
                t_cluster = t;
                best_cluster = v;
            }
        }
    }
    cudaStreamSynchronize(s->stream);
    if (ok) cudaMemcpy(s->flag, &flag0, sizeof(int), cudaMemcpyHostToDevice);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int k = 0; k < 2; ++k) {
        tmp_free(tf[k], fb);
        tmp_free(tb[k], bb);
    }
    cudaGetLastError();
    if (best_cluster >= 0 && t_cluster < t_graph && t_cluster < t_multi) {
        if ((size_t)cluster_blocks(best_cluster) > s->partial_blocks) {
            double* p = (double*)s->dalloc((size_t)cluster_blocks(best_cluster) * (s->D + 2) * sizeof(double));
            if (!p) return fail(LBM_ENOMEM, "diagnostics partial buffer");
            s->partial = p;
            s->partial_blocks = cluster_blocks(best_cluster);
        }
        s->cluster_v = best_cluster;
        s->multi_k = K;
    } else if (t_multi < t_graph) {
        s->multi_k = K;
    }
    return LBM_OK;
}

lbm_status autotune(lbm_sim* s) {
    if (s->opts.inplace) {  // one kernel pair, one thread per site
        s->var = kInplaceVariant;
        s->chunk = 0;
        return ensure_partial(s, s->var, s->chunk);
    }
    if (s->opts.model == LBM_MODEL_STANDARD) {  // one kernel, planes per block fixed
        s->var = kStdVariant;
        s->chunk = s->opts.chunk > 0 ? s->opts.chunk : 32;
        return ensure_partial(s, s->var, s->chunk);
    }
    // Lattices that share a result: same dimension, storage, extents,
    // boundary and set of kernels that implement their settings (plain;
    // force or MRT without walls; walls or the small-T recovery).  A forced
    // tile or chunk is not looked up.
    const int kernels = ext_ok(s) ? 2 : (walls_ok(s) ? 3 : (generic_only(s) ? 1 : 0));
    auto key = std::make_tuple(s->D, s->dtype * 4 + kernels, (int)s->bc, s->nx, s->ny, s->nz);
    const bool forced_cfg = s->opts.tile >= 0 || s->opts.chunk > 0;
    if (!forced_cfg) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            s->var = it->second.first;
            s->chunk = it->second.second;
            return ensure_partial(s, s->var, s->chunk);
        }
    }
    int nv = n_variants(s->D);
    std::vector<int> vars;
    if (s->opts.tile >= 0 && variant_allowed(s, s->opts.tile) &&
        (s->opts.tile < nv || tma_applicable(s, s->opts.tile))) {
        vars.push_back(s->opts.tile);
    } else {
        for (int v = 0; v < nv; ++v)
            if (variant_allowed(s, v)) vars.push_back(v);
        for (int k = 0; k < n_tma_variants(s->D); ++k)
            if (tma_applicable(s, kTmaBase + k)) vars.push_back(kTmaBase + k);
        for (int k = 0; k < n_pair_variants(s->D); ++k)
            if (tma_applicable(s, kPairBase + k)) vars.push_back(kPairBase + k);
        for (int k = 0; k < n_own_variants(s->D); ++k)
            if (tma_applicable(s, kOwnBase + k)) vars.push_back(kOwnBase + k);
    }
    std::vector<int> chunks = s->opts.chunk > 0 ? std::vector<int>{s->opts.chunk} : chunk_candidates(s);
    if (vars.size() * chunks.size() == 1) {
        s->var = vars[0];
        s->chunk = chunks[0];
        return ensure_partial(s, s->var, s->chunk);
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bv = vars[0], bc = chunks[0];
    // Candidates read the current state and write the other buffer only, so
    // the simulation state is untouched; no diagnostics, no flag updates
    // beyond what a real step would raise.
    for (int v : vars) {
        for (int c : chunks) {
            StepArgs a = base_args(s);
            a.chunk = c;
            a.write_state = 1;
            a.want_diag = 0;
            size_t smem = step_smem(s->D, s->dtype, v);
            if (smem > 227 * 1024) continue;
            if (launch_variant(s, v, a, s->cur) != LBM_OK) {
                cudaGetLastError();
                continue;
            }
            const int reps = 3;
            CK(cudaEventRecord(e0, s->stream));
            for (int r = 0; r < reps; ++r) {
                lbm_status st = launch_variant(s, v, a, s->cur);
                if (st != LBM_OK) return st;
            }
            CK(cudaEventRecord(e1, s->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bv = v;
                bc = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->var = bv;
    s->chunk = bc;
    if (!forced_cfg) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[key] = {bv, bc};
    }
    return ensure_partial(s, s->var, s->chunk);
}

lbm_status ensure_tuned(lbm_sim* s) {
    if (s->var >= 0) return LBM_OK;
    return autotune(s);
}

lbm_status build_graph(lbm_sim* s, int parity, int steps) {
    cudaGraph_t g;
    int saved = s->cur;
    s->cur = parity;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    lbm_status st = LBM_OK;
    for (int k = 0; k < steps && st == LBM_OK; ++k) st = launch_one_step(s, s->opts.diagnostics != 0);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    s->cur = saved;
    if (st != LBM_OK) return st;
    CK(e);
    e = cudaGraphInstantiate(&s->graph[parity], g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return LBM_OK;
}

// The captured graphs hold the step arguments of their capture: after a
// setting changes they are dropped and captured again at the next step.
void drop_graphs(lbm_sim* s) {
    for (int k = 0; k < 2; ++k)
        if (s->graph[k]) {
            cudaGraphExecDestroy(s->graph[k]);
            s->graph[k] = nullptr;
        }
}

// A setting only the generic kernel implements (walls, force, MRT) sends a
// lattice tuned onto another kernel back to the autotuner.
void retune_if_needed(lbm_sim* s) {
    if ((s->var >= 0 && !variant_allowed(s, s->var)) || (s->cluster_v >= 0 && generic_only(s))) {
        s->var = -1;
        s->multi_k = 0;
        s->cluster_v = -1;
    }
}

lbm_status check_flag(lbm_sim* s) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (h & 4) return fail(LBM_ETIMEOUT, "a bounded device-side wait for a tile copy gave up");
    if (h & 1) return fail(LBM_EUNSTABLE, "state became non-physical (rho <= 0 or not finite)");
    return LBM_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

void lbm_default_opts(lbm_opts* o) {
    std::memset(o, 0, sizeof(*o));
    o->dtype = LBM_F64;
    o->thermal = 0;
    o->device = 0;
    o->stream = nullptr;
    o->tile = -1;
    o->chunk = 0;
    o->steps_per_launch = 0;
    o->diagnostics = 1;
    o->use_graphs = 1;
}

const char* lbm_last_error(void) { return g_err.c_str(); }

const char* lbm_version(void) { return "bump-lbm-gb300 0.1 (sm_103a)"; }

lbm_status lbm_create(int dim, int nx, int ny, int nz, double tau, double T0, lbm_bc bc, lbm_sim** out) {
    lbm_opts o;
    lbm_default_opts(&o);
    return lbm_create_ex(dim, nx, ny, nz, tau, T0, bc, &o, out);
}

lbm_status lbm_create_ex(int dim, int nx, int ny, int nz, double tau, double T0, lbm_bc bc, const lbm_opts* opts,
                         lbm_sim** out) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (dim < 1 || dim > 3) return fail(LBM_EINVAL, "dim must be 1, 2 or 3");
    if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_EINVAL, "extents must be >= 1");
    if ((dim < 2 && ny != 1) || (dim < 3 && nz != 1)) return fail(LBM_EINVAL, "unused extents must be 1");
    if (!(tau > 0) || !(T0 > 0)) return fail(LBM_EINVAL, "tau and T0 must be > 0");
    if (bc != LBM_BC_PERIODIC && bc != LBM_BC_FIXED_STATE && bc != LBM_BC_WALLS)
        return fail(LBM_EINVAL, "unknown boundary");
    if (bc == LBM_BC_WALLS && dim < 2) return fail(LBM_EINVAL, "walls need dim 2 or 3");
    lbm_opts o;
    if (opts)
        o = *opts;
    else
        lbm_default_opts(&o);
    if (o.dtype < LBM_F64 || o.dtype > LBM_BF16_SHIFTED) return fail(LBM_EINVAL, "unknown dtype");
    if ((o.alloc == nullptr) != (o.free == nullptr)) return fail(LBM_EINVAL, "alloc and free go together");
    if (o.model != LBM_MODEL_BUMP && o.model != LBM_MODEL_STANDARD) return fail(LBM_EINVAL, "unknown model");
    if (o.model == LBM_MODEL_STANDARD && (bc != LBM_BC_PERIODIC || ny > 65535 || nz > 65535))
        return fail(LBM_EINVAL, "the standard comparator runs on periodic lattices with ny, nz <= 65535");
    if (o.halo != 0 && o.halo != 2) return fail(LBM_EINVAL, "halo must be 0 or 2");
    if (o.inplace != 0 && o.inplace != 1) return fail(LBM_EINVAL, "inplace must be 0 or 1");
    if (o.cluster < -1 || o.cluster > n_cluster_variants())
        return fail(LBM_EINVAL, "cluster must be -1, 0 or 1 + a cluster variant");
    if (o.inplace && (bc != LBM_BC_PERIODIC || o.model != LBM_MODEL_BUMP || o.halo ||
                      (o.dtype != LBM_F64 && o.dtype != LBM_F32)))
        return fail(LBM_EINVAL, "the in-place step: bump scheme, periodic, FP64 or FP32 storage, no halo");
    if (o.halo) {
        if (dim < 2 || bc == LBM_BC_WALLS || o.model != LBM_MODEL_BUMP)
            return fail(LBM_EINVAL, "halo planes: the bump scheme in 2D/3D, periodic or fixed-state in x");
        if ((dim == 3 ? nz : ny) < 2 * o.halo + 1)
            return fail(LBM_EINVAL, "halo planes: the slowest axis needs at least one plane besides the halos");
    }
    long long N = (long long)nx * ny * nz;
    int Q = q_of(dim), NB = nb_of(dim);
    if ((long long)Q * N >= (1LL << 40)) return fail(LBM_EINVAL, "lattice too large");

    lbm_sim* s = new lbm_sim();
    s->D = dim;
    s->Q = Q;
    s->NB = NB;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->N = N;
    s->rows = (long long)ny * nz;
    s->tau = tau;
    s->T0 = T0;
    s->bc = bc;
    s->opts = o;
    s->dtype = (int)o.dtype;
    s->device = o.device;
    DeviceGuard dg(s->device);
    cudaError_t e;
    if (o.stream) {
        s->stream = (cudaStream_t)o.stream;
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return fail(LBM_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        s->own_stream = true;
    }
    size_t fb = fbytes_of(s->dtype), rb = rbytes_of(s->dtype);
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        // in place: one population buffer, both parities refer to it
        s->f[k] = (o.inplace && k == 1) ? s->f[0] : s->dalloc((size_t)Q * N * fb);
        s->b[k] = s->dalloc((size_t)NB * N * rb);
        ok = s->f[k] && s->b[k];
    }
    if (ok && o.inplace) {
        s->aux = s->dalloc((size_t)(dim + NB) * N * rb);
        ok = s->aux != nullptr;
    }
    if (ok && bc == LBM_BC_FIXED_STATE) {
        s->gf = s->dalloc((size_t)2 * Q * s->rows * rb);
        s->gb = s->dalloc((size_t)2 * NB * s->rows * rb);
        s->gaux = s->dalloc((size_t)2 * (dim + NB) * s->rows * rb);
        ok = s->gf && s->gb && s->gaux;
    }
    if (ok) {
        s->ticket = (unsigned int*)s->dalloc(64);
        s->step_ctr = (long long*)s->dalloc(64);
        s->flag = (int*)s->dalloc(64);
        s->diag_out = (double*)s->dalloc(64);
        s->hist = (double*)s->dalloc((size_t)kHistCap * (dim + 3) * sizeof(double));
        ok = s->ticket && s->step_ctr && s->flag && s->diag_out && s->hist;
    }
    if (!ok) {
        s->release();
        delete s;
        return fail(LBM_ENOMEM, "device allocation failed");
    }
    cudaMemsetAsync(s->ticket, 0, 64, s->stream);
    cudaMemsetAsync(s->step_ctr, 0, 64, s->stream);
    cudaMemsetAsync(s->flag, 0, 64, s->stream);
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        s->release();
        delete s;
        return fail(LBM_ECUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    *out = s;
    return LBM_OK;
}

void lbm_destroy(lbm_sim* s) {
    if (!s) return;
    DeviceGuard dg(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->release();
    delete s;
}

static lbm_status ensure_fields(lbm_sim* s) {
    if (s->fields) return LBM_OK;
    s->fields = (double*)s->dalloc((size_t)(s->D + 2) * s->N * sizeof(double));
    if (!s->fields) return fail(LBM_ENOMEM, "fields buffer");
    return LBM_OK;
}

lbm_status lbm_init(lbm_sim* s, const lbm_fields_in* in) {
    if (!s || !in || !in->rho || !in->u || !in->T) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(s->device);
    const long long N = s->N;
    lbm_status st = ensure_fields(s);
    if (st != LBM_OK) return st;
    double* rho = s->fields;
    double* u = rho + N;
    double* T = u + (size_t)s->D * N;
    CK(cudaMemcpyAsync(rho, in->rho, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(T, in->T, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    // positivity of rho and T checked on the device while u is copied; the
    // state is touched only once the check has passed
    int* bad = s->flag + 1;
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s->stream));
    CK(launch_check_fields(rho, T, N, bad, s->stream));
    CK(cudaMemcpyAsync(u, in->u, (size_t)s->D * N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (hbad) return fail(LBM_EINVAL, "rho and T must be positive");
    s->cur = 0;
    if (s->opts.model == LBM_MODEL_STANDARD) {
        CK(launch_std_init(s->D, s->dtype, rho, u, T, s->f[0], N, s->stream));
        for (int k = 0; k < 2; ++k)  // no variance: keep both buffers defined
            CK(cudaMemsetAsync(s->b[k], 0, (size_t)s->NB * N * rbytes_of(s->dtype), s->stream));
    } else {
        CK(launch_init(s->D, s->dtype, rho, u, T, s->f[0], s->b[0], N, s->stream));
    }
    if (s->bc == LBM_BC_FIXED_STATE)
        CK(launch_reservoir(s->D, s->dtype, rho, u, T, s->nx, s->rows, N, s->gf, s->gb, s->gaux, s->stream));
    CK(cudaMemsetAsync(s->step_ctr, 0, 64, s->stream));
    CK(cudaMemsetAsync(s->flag, 0, 64, s->stream));
    CK(cudaMemsetAsync(s->ticket, 0, 64, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->nstep = 0;
    return LBM_OK;
}

lbm_status lbm_set_force(lbm_sim* s, const double* a) {
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (s->opts.inplace && a) return fail(LBM_EINVAL, "the in-place step has no body force");
    if (s->opts.model == LBM_MODEL_STANDARD && a) return fail(LBM_EINVAL, "the standard comparator has no body force");
    double v[3] = {0, 0, 0};
    if (a)
        for (int c = 0; c < s->D; ++c) {
            if (!std::isfinite(a[c])) return fail(LBM_EINVAL, "acceleration must be finite");
            v[c] = a[c];
        }
    DeviceGuard dg(s->device);
    // graphs captured the old arguments; wait for launches that use them
    CK(cudaStreamSynchronize(s->stream));
    for (int c = 0; c < 3; ++c) s->acc[c] = v[c];
    s->forced = v[0] != 0 || v[1] != 0 || v[2] != 0;
    drop_graphs(s);
    retune_if_needed(s);
    return LBM_OK;
}

lbm_status lbm_set_mrt(lbm_sim* s, double s3, double s4) {
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    const bool on = s3 > 0 || s4 > 0;
    if (on && s->opts.inplace) return fail(LBM_EINVAL, "the in-place step runs the SRT collision");
    if (on && (s->D != 3 || s->opts.model != LBM_MODEL_BUMP))
        return fail(LBM_EINVAL, "the MRT collision needs the D3Q19 bump scheme");
    if (on && !(s3 > 0 && s3 < 2 && s4 > 0 && s4 < 2)) return fail(LBM_EINVAL, "MRT rates must lie in (0, 2)");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));  // graphs captured the old arguments
    s->mrt = on;
    s->mrt_s[0] = on ? s3 : 0;
    s->mrt_s[1] = on ? s4 : 0;
    drop_graphs(s);
    retune_if_needed(s);
    return LBM_OK;
}

lbm_status lbm_set_small_t(lbm_sim* s, double kappa) {
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (s->opts.inplace && kappa > 0) return fail(LBM_EINVAL, "the in-place step has no FP64 small-T recovery");
    if (!(kappa >= 0) || !std::isfinite(kappa)) return fail(LBM_EINVAL, "kappa must be finite and >= 0");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));  // graphs captured the old arguments
    s->small_t = kappa;
    drop_graphs(s);
    retune_if_needed(s);
    return LBM_OK;
}

lbm_status lbm_set_debug(lbm_sim* s, int flags) {
    if (!s) return fail(LBM_EINVAL, "NULL sim");
    if (flags & ~LBM_DEBUG_MISSING_COPY) return fail(LBM_EINVAL, "unknown debug flag");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));
    s->debug = flags;
    drop_graphs(s);  // captured launches hold the old arguments
    return LBM_OK;
}

lbm_status lbm_set_wall_velocity(lbm_sim* s, const double* lo, const double* hi) {
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (s->bc != LBM_BC_WALLS) return fail(LBM_EINVAL, "wall velocities need LBM_BC_WALLS");
    double v[2][3] = {{0, 0, 0}, {0, 0, 0}};
    const double* in[2] = {lo, hi};
    for (int w = 0; w < 2; ++w)
        if (in[w])
            for (int c = 0; c < s->D; ++c) {
                if (!std::isfinite(in[w][c])) return fail(LBM_EINVAL, "wall velocity must be finite");
                v[w][c] = in[w][c];
            }
    if (v[0][s->D - 1] != 0 || v[1][s->D - 1] != 0)
        return fail(LBM_EINVAL, "wall velocities must be tangential (zero along the last axis)");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));  // graphs captured the old arguments
    bool moving = false;
    for (int w = 0; w < 2; ++w)
        for (int c = 0; c < 3; ++c) {
            s->uw[w][c] = v[w][c];
            moving = moving || v[w][c] != 0;
        }
    s->walls_moving = moving;
    drop_graphs(s);
    return LBM_OK;
}

lbm_status lbm_step(lbm_sim* s, long n) {
    if (!s) return fail(LBM_EINVAL, "NULL sim");
    if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
    if (n == 0) return LBM_OK;
    DeviceGuard dg(s->device);
    lbm_status st = ensure_tuned(s);
    if (st != LBM_OK) return st;
    const bool diag = s->opts.diagnostics != 0;
    const int K = s->graph_steps;
    long done = 0;
    if (s->multi_k == 0) {
        st = tune_multi(s);
        if (st != LBM_OK) return st;
    }
    if (s->multi_k > 1) {
        // D1: several steps per cooperative launch
        void* f[2] = {s->f[0], s->f[1]};
        void* b[2] = {s->b[0], s->b[1]};
        while (done < n) {
            const int k = (int)std::min<long>(s->multi_k, n - done);
            st = launch_multi(s, k, diag, f, b);
            if (st != LBM_OK) return st;
            if (k & 1) s->cur = 1 - s->cur;
            done += k;
        }
        s->nstep += n;
        return LBM_OK;
    }
    if (s->opts.use_graphs && s->stream != nullptr && n >= 2) {
        if (K == 0) {
            // graph length: more launches per replay for small lattices
            int steps = (s->N * s->Q < (1LL << 22)) ? 32 : 2;
            s->graph_steps = steps;
        }
        const int GK = s->graph_steps;
        while (n - done >= GK) {
            if (!s->graph[s->cur]) {
                st = build_graph(s, s->cur, GK);
                if (st != LBM_OK) return st;
            }
            CK(cudaGraphLaunch(s->graph[s->cur], s->stream));
            if (GK % 2) s->cur = 1 - s->cur;
            done += GK;
        }
    }
    for (; done < n; ++done) {
        st = launch_one_step(s, diag);
        if (st != LBM_OK) return st;
    }
    s->nstep += n;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_sim* s) {
    if (!s) return fail(LBM_EINVAL, "NULL sim");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));
    return check_flag(s);
}

long lbm_step_count(const lbm_sim* s) { return s ? s->nstep : -1; }

lbm_status lbm_launch_config(const lbm_sim* s, int* tile, int* chunk, const char** kernel) {
    if (!s) return fail(LBM_EINVAL, "NULL simulation");
    const bool cl = s->multi_k > 1 && s->cluster_v >= 0;
    if (tile) *tile = cl ? kClusterBase + s->cluster_v : s->var;
    if (chunk) *chunk = s->var >= 0 ? (s->multi_k > 1 ? s->multi_k : s->chunk) : -1;
    if (kernel)
        *kernel = s->var < 0 ? ""
                             : (cl ? "step_cluster_kernel"
                                   : (s->multi_k > 1 ? "step_multi_kernel" : kernel_name(s->D, s->var)));
    return LBM_OK;
}

lbm_status lbm_flags(lbm_sim* s, int* flags) {
    if (!s || !flags) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(s->device);
    CK(cudaMemcpyAsync(flags, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_moments(lbm_sim* s, lbm_fields_out* out) {
    if (!s || !out) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(s->device);
    lbm_status st = ensure_tuned(s);
    if (st != LBM_OK) return st;
    st = ensure_fields(s);
    if (st != LBM_OK) return st;
    StepArgs a = base_args(s);
    a.write_state = 0;
    a.want_diag = 0;
    a.mout = s->fields;
    st = launch_variant(s, s->var, a, s->cur);
    if (st != LBM_OK) return st;
    const long long N = s->N;
    if (out->rho) CK(cudaMemcpyAsync(out->rho, s->fields, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (out->u)
        CK(cudaMemcpyAsync(out->u, s->fields + N, (size_t)s->D * N * sizeof(double), cudaMemcpyDeviceToHost,
                           s->stream));
    if (out->T)
        CK(cudaMemcpyAsync(out->T, s->fields + (size_t)(1 + s->D) * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                           s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return check_flag(s);
}

lbm_status lbm_diagnostics(lbm_sim* s, double* out) {
    if (!s || !out) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(s->device);
    lbm_status st = ensure_tuned(s);
    if (st != LBM_OK) return st;
    StepArgs a = base_args(s);
    a.write_state = 0;
    a.want_diag = 1;
    a.diag_out = s->diag_out;
    a.hist = nullptr;
    st = launch_variant(s, s->var, a, s->cur);
    if (st != LBM_OK) return st;
    CK(cudaMemcpyAsync(out, s->diag_out, (size_t)(s->D + 2) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return check_flag(s);
}

lbm_status lbm_diagnostics_history(lbm_sim* s, double* out, int cap, int* count) {
    if (!s || !out || !count || cap < 0) return fail(LBM_EINVAL, "bad argument");
    DeviceGuard dg(s->device);
    long long ctr = 0;
    CK(cudaMemcpyAsync(&ctr, s->step_ctr, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const int rec = s->D + 3;
    long long avail = ctr < kHistCap ? ctr : kHistCap;
    long long n = avail < cap ? avail : cap;
    std::vector<double> h((size_t)kHistCap * rec);
    CK(cudaMemcpy(h.data(), s->hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (long long k = 0; k < n; ++k) {
        long long idx = (ctr - n + k) % kHistCap;
        std::memcpy(out + k * rec, h.data() + idx * rec, rec * sizeof(double));
    }
    *count = (int)n;
    return LBM_OK;
}

lbm_status lbm_last_diagnostics(lbm_sim* s, double* out) {
    if (!s || !out) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(s->device);
    // the step counter and the status flag in one wait, then the record
    long long ctr = 0;
    int h = 0;
    CK(cudaMemcpyAsync(&ctr, s->step_ctr, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(&h, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (ctr <= 0) return fail(LBM_EINVAL, "no diagnostics recorded yet");
    const int rec = s->D + 3;
    CK(cudaMemcpyAsync(out, s->hist + ((ctr - 1) % kHistCap) * rec, rec * sizeof(double), cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (h & 4) return fail(LBM_ETIMEOUT, "a bounded device-side wait for a tile copy gave up");
    if (h & 1) return fail(LBM_EUNSTABLE, "state became non-physical (rho <= 0 or not finite)");
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_sim* s, double* f, double* b) {
    if (!s) return fail(LBM_EINVAL, "NULL sim");
    DeviceGuard dg(s->device);
    const long long N = s->N;
    double* tmp = (double*)s->dalloc((size_t)(s->Q + s->NB) * N * sizeof(double));
    if (!tmp) return fail(LBM_ENOMEM, "state staging buffer");
    lbm_status st = LBM_OK;
    cudaError_t e = launch_get_state(s->D, s->dtype, s->f[s->cur], s->b[s->cur], tmp, tmp + (size_t)s->Q * N, N,
                                     s->stream);
    if (e == cudaSuccess && s->opts.inplace && s->cur == 1) {
        // in place after an odd number of steps: the arrived populations
        StepArgs a = base_args(s);
        e = launch_aa_get_state(s->D, s->dtype, a, tmp, s->stream);
    }
    if (e == cudaSuccess && f)
        e = cudaMemcpyAsync(f, tmp, (size_t)s->Q * N * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && b)
        e = cudaMemcpyAsync(b, tmp + (size_t)s->Q * N, (size_t)s->NB * N * sizeof(double), cudaMemcpyDeviceToHost,
                            s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = fail(LBM_ECUDA, std::string("get_state: ") + cudaGetErrorString(e));
    // release the staging buffer
    for (size_t k = 0; k < s->allocs.size(); ++k)
        if (s->allocs[k].first == tmp) {
            if (s->opts.alloc)
                s->opts.free(tmp, s->allocs[k].second, s->opts.alloc_ctx);
            else
                cudaFree(tmp);
            s->allocs.erase(s->allocs.begin() + k);
            break;
        }
    return st;
}

lbm_status lbm_set_state(lbm_sim* s, const double* f, const double* b) {
    if (!s) return fail(LBM_EINVAL, "NULL sim");
    if (s->opts.inplace && s->cur == 1) {
        // the buffer holds arrived populations: a full state restarts it in
        // the emitted layout
        if (!f || !b) return fail(LBM_EINVAL, "an in-place simulation after an odd step count takes f and b together");
        s->cur = 0;
    }
    DeviceGuard dg(s->device);
    const long long N = s->N;
    double* tmp = (double*)s->dalloc((size_t)(s->Q + s->NB) * N * sizeof(double));
    if (!tmp) return fail(LBM_ENOMEM, "state staging buffer");
    cudaError_t e = cudaSuccess;
    if (f) e = cudaMemcpyAsync(tmp, f, (size_t)s->Q * N * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && b)
        e = cudaMemcpyAsync(tmp + (size_t)s->Q * N, b, (size_t)s->NB * N * sizeof(double), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess)
        e = launch_set_state(s->D, s->dtype, s->f[s->cur], s->b[s->cur], f ? tmp : nullptr,
                             b ? tmp + (size_t)s->Q * N : nullptr, N, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    lbm_status st = e == cudaSuccess ? LBM_OK : fail(LBM_ECUDA, std::string("set_state: ") + cudaGetErrorString(e));
    for (size_t k = 0; k < s->allocs.size(); ++k)
        if (s->allocs[k].first == tmp) {
            if (s->opts.alloc)
                s->opts.free(tmp, s->allocs[k].second, s->opts.alloc_ctx);
            else
                cudaFree(tmp);
            s->allocs.erase(s->allocs.begin() + k);
            break;
        }
    return st;
}

// Checkpoint file: header, then the emitted planes in the storage dtype, then
// the reservoirs (fixed-state boundary only).  `model` is lbm_opts.model: a
// bump-scheme state and a comparator state have the same planes but do not
// mean the same thing, so a load across models is refused.
struct CkptHeader {
    char magic[8];
    int D, nx, ny, nz, dtype, bc, thermal, model;
    double tau, T0;
    long long nstep;
};

lbm_status lbm_save(lbm_sim* s, const char* path) {
    if (!s || !path) return fail(LBM_EINVAL, "NULL argument");
    if (s->opts.inplace && s->cur == 1)
        return fail(LBM_EINVAL, "an in-place simulation is saved after an even number of steps");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));
    const long long N = s->N;
    size_t fb = (size_t)s->Q * N * fbytes_of(s->dtype), bb = (size_t)s->NB * N * rbytes_of(s->dtype);
    std::vector<char> buf(fb + bb);
    CK(cudaMemcpy(buf.data(), s->f[s->cur], fb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(buf.data() + fb, s->b[s->cur], bb, cudaMemcpyDeviceToHost));
    size_t rb = rbytes_of(s->dtype);
    size_t g1 = 0, g2 = 0, g3 = 0;
    std::vector<char> gbuf;
    if (s->bc == LBM_BC_FIXED_STATE) {
        g1 = (size_t)2 * s->Q * s->rows * rb;
        g2 = (size_t)2 * s->NB * s->rows * rb;
        g3 = (size_t)2 * (s->D + s->NB) * s->rows * rb;
        gbuf.resize(g1 + g2 + g3);
        CK(cudaMemcpy(gbuf.data(), s->gf, g1, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(gbuf.data() + g1, s->gb, g2, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(gbuf.data() + g1 + g2, s->gaux, g3, cudaMemcpyDeviceToHost));
    }
    CkptHeader h{};
    std::memcpy(h.magic, "BUMPLBM1", 8);
    h.D = s->D;
    h.nx = s->nx;
    h.ny = s->ny;
    h.nz = s->nz;
    h.dtype = s->dtype;
    h.bc = s->bc;
    h.thermal = s->opts.thermal;
    h.model = s->opts.model;
    h.tau = s->tau;
    h.T0 = s->T0;
    h.nstep = s->nstep;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(LBM_EIO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size() &&
              (gbuf.empty() || std::fwrite(gbuf.data(), 1, gbuf.size(), fp) == gbuf.size());
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(LBM_EIO, std::string("write failed: ") + path);
    return LBM_OK;
}

lbm_status lbm_load(lbm_sim* s, const char* path) {
    if (!s || !path) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(s->device);
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(LBM_EIO, std::string("cannot open ") + path);
    CkptHeader h{};
    if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, "BUMPLBM1", 8) != 0) {
        std::fclose(fp);
        return fail(LBM_EIO, "not a checkpoint file");
    }
    if (h.D != s->D || h.nx != s->nx || h.ny != s->ny || h.nz != s->nz || h.dtype != s->dtype || h.bc != s->bc) {
        std::fclose(fp);
        return fail(LBM_EINVAL, "checkpoint does not match this simulation");
    }
    if (h.model != s->opts.model) {
        std::fclose(fp);
        return fail(LBM_EINVAL, "checkpoint holds the state of another model (lbm_opts.model)");
    }
    // the same checks lbm_create_ex applies: a corrupt or foreign file must
    // not set a meaningless omega = 1/(tau + 1/2)
    if (!std::isfinite(h.tau) || !(h.tau > 0) || !std::isfinite(h.T0) || !(h.T0 > 0) || (h.thermal != 0 && h.thermal != 1) ||
        h.nstep < 0) {
        std::fclose(fp);
        return fail(LBM_EIO, "checkpoint header holds invalid parameters (tau, T0, thermal or step count)");
    }
    const long long N = s->N;
    size_t fb = (size_t)s->Q * N * fbytes_of(s->dtype), bb = (size_t)s->NB * N * rbytes_of(s->dtype);
    std::vector<char> buf(fb + bb);
    bool ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    size_t rb = rbytes_of(s->dtype);
    std::vector<char> gbuf;
    size_t g1 = 0, g2 = 0, g3 = 0;
    if (ok && s->bc == LBM_BC_FIXED_STATE) {
        g1 = (size_t)2 * s->Q * s->rows * rb;
        g2 = (size_t)2 * s->NB * s->rows * rb;
        g3 = (size_t)2 * (s->D + s->NB) * s->rows * rb;
        gbuf.resize(g1 + g2 + g3);
        ok = std::fread(gbuf.data(), 1, gbuf.size(), fp) == gbuf.size();
    }
    std::fclose(fp);
    if (!ok) return fail(LBM_EIO, "truncated checkpoint");
    CK(cudaStreamSynchronize(s->stream));
    if (s->opts.inplace) s->cur = 0;  // the file holds the emitted layout
    CK(cudaMemcpy(s->f[s->cur], buf.data(), fb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->b[s->cur], buf.data() + fb, bb, cudaMemcpyHostToDevice));
    if (!gbuf.empty()) {
        CK(cudaMemcpy(s->gf, gbuf.data(), g1, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(s->gb, gbuf.data() + g1, g2, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(s->gaux, gbuf.data() + g1 + g2, g3, cudaMemcpyHostToDevice));
    }
    s->opts.thermal = h.thermal;
    s->tau = h.tau;
    s->T0 = h.T0;
    s->nstep = (long)h.nstep;
    long long ctr = h.nstep;
    CK(cudaMemcpy(s->step_ctr, &ctr, sizeof(ctr), cudaMemcpyHostToDevice));
    CK(cudaMemset(s->flag, 0, sizeof(int)));
    // a step that gave up (LBM_ETIMEOUT) left the reduction ticket counted short
    CK(cudaMemset(s->ticket, 0, 64));
    drop_graphs(s);
    return LBM_OK;
}

}  // extern "C"

// ---- domain decomposition: halo planes of slab simulations -----------------

namespace {

// One stored array of a state buffer as rows of the slowest axis: `rows`
// rows (planes of populations or of variance components), row pitch and
// the bytes of one lattice plane within a row.
struct SlabArrays {
    size_t f_pitch, f_plane, b_pitch, b_plane;
    int f_rows, b_rows;
};

SlabArrays slab_arrays(const lbm_sim* s) {
    SlabArrays A{};
    const size_t fb = fbytes_of(s->dtype), rb = rbytes_of(s->dtype);
    const size_t pstride = s->D == 3 ? (size_t)s->nx * s->ny : (size_t)s->nx;
    A.f_rows = s->Q;
    A.f_pitch = (size_t)s->N * fb;
    A.f_plane = pstride * fb;
    // variance: component-major planes, or (3D, 32/16-bit storage) three
    // planes of component pairs interleaved per site
    const bool paired = s->D == 3 && s->dtype != DT_F64;
    A.b_rows = paired ? s->NB / 2 : s->NB;
    A.b_pitch = (size_t)s->N * rb * (paired ? 2 : 1);
    A.b_plane = pstride * rb * (paired ? 2 : 1);
    return A;
}

// Copy `np` planes of the slowest axis starting at plane p_src of sim `a`'s
// current state into planes starting at p_dst of sim `b`'s current state
// (populations and variance), on `st`.
cudaError_t copy_planes(const lbm_sim* a, int p_src, lbm_sim* b, int p_dst, int np, cudaStream_t st) {
    const SlabArrays A = slab_arrays(a);
    const char* fs = static_cast<const char*>(a->f[a->cur]);
    char* fd = static_cast<char*>(b->f[b->cur]);
    cudaError_t e = cudaMemcpy2DAsync(fd + p_dst * A.f_plane, A.f_pitch, fs + p_src * A.f_plane, A.f_pitch,
                                      np * A.f_plane, A.f_rows, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return e;
    const char* bs = static_cast<const char*>(a->b[a->cur]);
    char* bd = static_cast<char*>(b->b[b->cur]);
    return cudaMemcpy2DAsync(bd + p_dst * A.b_plane, A.b_pitch, bs + p_src * A.b_plane, A.b_pitch, np * A.b_plane,
                             A.b_rows, cudaMemcpyDefault, st);
}

int slab_planes(const lbm_sim* s) { return s->D == 3 ? s->nz : s->ny; }

}  // namespace

extern "C" {

size_t lbm_halo_bytes(const lbm_sim* s) {
    if (!s || !s->opts.halo) return 0;
    const SlabArrays A = slab_arrays(s);
    const int h = s->opts.halo;
    return (size_t)h * (A.f_rows * A.f_plane + A.b_rows * A.b_plane);
}

lbm_status lbm_halo_pack(lbm_sim* s, int side, void* dst) {
    if (!s || !dst) return fail(LBM_EINVAL, "NULL argument");
    if (!s->opts.halo) return fail(LBM_EINVAL, "the simulation has no halo planes (lbm_opts.halo)");
    if (side != 0 && side != 1) return fail(LBM_EINVAL, "side must be 0 (low) or 1 (high)");
    DeviceGuard dg(s->device);
    const SlabArrays A = slab_arrays(s);
    const int h = s->opts.halo, n = slab_planes(s);
    const int p = side == 0 ? h : n - 2 * h;  // the outermost owned planes on that side
    const char* fs = static_cast<const char*>(s->f[s->cur]);
    const char* bs = static_cast<const char*>(s->b[s->cur]);
    char* d = static_cast<char*>(dst);
    // message: the h planes of every population row, then of every variance row
    CK(cudaMemcpy2DAsync(d, h * A.f_plane, fs + p * A.f_plane, A.f_pitch, h * A.f_plane, A.f_rows,
                         cudaMemcpyDefault, s->stream));
    CK(cudaMemcpy2DAsync(d + (size_t)A.f_rows * h * A.f_plane, h * A.b_plane, bs + p * A.b_plane, A.b_pitch,
                         h * A.b_plane, A.b_rows, cudaMemcpyDefault, s->stream));
    return LBM_OK;
}

lbm_status lbm_halo_unpack(lbm_sim* s, int side, const void* src) {
    if (!s || !src) return fail(LBM_EINVAL, "NULL argument");
    if (!s->opts.halo) return fail(LBM_EINVAL, "the simulation has no halo planes (lbm_opts.halo)");
    if (side != 0 && side != 1) return fail(LBM_EINVAL, "side must be 0 (low) or 1 (high)");
    DeviceGuard dg(s->device);
    const SlabArrays A = slab_arrays(s);
    const int h = s->opts.halo, n = slab_planes(s);
    const int p = side == 0 ? 0 : n - h;  // the halo planes on that side
    char* fd = static_cast<char*>(s->f[s->cur]);
    char* bd = static_cast<char*>(s->b[s->cur]);
    const char* m = static_cast<const char*>(src);
    CK(cudaMemcpy2DAsync(fd + p * A.f_plane, A.f_pitch, m, h * A.f_plane, h * A.f_plane, A.f_rows,
                         cudaMemcpyDefault, s->stream));
    CK(cudaMemcpy2DAsync(bd + p * A.b_plane, A.b_pitch, m + (size_t)A.f_rows * h * A.f_plane, h * A.b_plane,
                         h * A.b_plane, A.b_rows, cudaMemcpyDefault, s->stream));
    return LBM_OK;
}

lbm_status lbm_halo_exchange(lbm_sim* const* sims, int k) {
    if (!sims || k < 1) return fail(LBM_EINVAL, "need at least one slab");
    for (int i = 0; i < k; ++i) {
        if (!sims[i]) return fail(LBM_EINVAL, "NULL slab");
        const lbm_sim* a = sims[i];
        const lbm_sim* b = sims[0];
        if (!a->opts.halo) return fail(LBM_EINVAL, "a slab has no halo planes (lbm_opts.halo)");
        if (a->D != b->D || a->nx != b->nx || (a->D == 3 && a->ny != b->ny) || a->dtype != b->dtype ||
            a->opts.halo != b->opts.halo)
            return fail(LBM_EINVAL, "slabs differ in dimension, cross-section, storage or halo depth");
    }
    // ordering: every slab's last step is complete (event on its stream)
    // before any copy out of it; the copies into slab j run on j's stream,
    // so its next step follows them; and the copies out of slab i finish
    // before i's step after next, which rewrites that buffer -- i's stream
    // waits for the other streams' events at the next exchange, and every
    // step is followed by one
    std::vector<cudaEvent_t> ev(k);
    for (int i = 0; i < k; ++i) {
        DeviceGuard dg(sims[i]->device);
        CK(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
        CK(cudaEventRecord(ev[i], sims[i]->stream));
    }
    lbm_status st = LBM_OK;
    for (int j = 0; j < k && st == LBM_OK; ++j) {
        lbm_sim* b = sims[j];
        DeviceGuard dg(b->device);
        const int lo = (j + k - 1) % k, hi = (j + 1) % k;
        const int h = b->opts.halo, nb = slab_planes(b);
        cudaError_t e = cudaStreamWaitEvent(b->stream, ev[lo], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev[hi], 0);
        // low halo of j <- the top owned planes of the slab below
        if (e == cudaSuccess) e = copy_planes(sims[lo], slab_planes(sims[lo]) - 2 * h, b, 0, h, b->stream);
        // high halo of j <- the bottom owned planes of the slab above
        if (e == cudaSuccess) e = copy_planes(sims[hi], h, b, nb - h, h, b->stream);
        if (e != cudaSuccess) st = fail(LBM_ECUDA, std::string("halo exchange: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < k; ++i) cudaEventDestroy(ev[i]);
    return st;
}

}  // extern "C"
