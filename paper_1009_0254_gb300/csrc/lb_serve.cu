// lb_serve.cu -- a request server with continuous batching.
//
// Simulations (lattice size, parameters, seed, number of steps) are submitted at any time
// from any host thread.  A scheduler thread admits them in arrival order, backfilling
// smaller ones, as device memory (an HBM budget, served from a stream-ordered memory pool)
// and slots allow, and advances every admitted simulation together: one persistent launch
// of the served step kernel per time step covers the tiles of all of them.  Steps are
// issued in chunks that end where the earliest admitted simulation finishes (capped), so
// that new arrivals join and finished ones leave between chunks; each simulation's state
// stays resident on the device from admission to completion.  A simulation's trajectory
// depends only on its own request: its step counter starts at 0 on admission and keys its
// Philox stream with its own seed, so a result is the same alone and in any mix.
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <cmath>
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

#include "lb_ens.cuh"
#include "lb_noise.cuh"
#include "lbfluct.h"

namespace lbf {

// per-slot descriptor (device)
struct SlotDesc {
    Grid g;
    float* buf[2];
    float2* xi;              // correlated noise (xi_4, xi_9) for the coming step, or null
    int ntx;                 // tiles along x
    long long k_start;       // server step counter at admission
};

struct ServeParams {
    const CUtensorMap* maps;     // [slot][2], maps of buffers 0 and 1
    const SlotDesc* desc;
    const RepRec* recs;
    const int* active;           // slots of this chunk
    const int* tile_begin;       // first tile of each active slot, ntiles at the end
    int nactive, ntiles;
    long long* kstep;            // server step counter K (device)
    unsigned int* done;
    int* err;
};

// tile of the served kernel: 64 x 16 nodes on 512 threads (measured against 64 x 8 on 256:
// faster on the request stream and on a large lattice alone, slower on a lone 256^2 one)
constexpr int SV_TX = 64, SV_TY = 16, SV_NT = 512;

// index of the active slot that owns `tile`: the last a with tile_begin[a] <= tile
__device__ __forceinline__ int find_owner(const int* __restrict__ tile_begin, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&tile_begin[mid]) <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// RS: the variant that also steps simulations with real-space correlated noise (launched
// for chunks that hold one; its extra path raises the register count)
template <int TX, int TY, int NT, bool RS>
__global__ void __launch_bounds__(NT, 1024 / NT) step_serve_kernel(const ServeParams p) {
    using TT = TmaTile<TX, TY, float>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* smem = reinterpret_cast<float*>(smem_raw);
    float* R = reinterpret_cast<float*>(smem_raw + 2 * TT::STAGE_BYTES);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(R + TT::RW * TT::RH);
    __shared__ int st_slot[2], st_x0[2], st_y0[2];
    __shared__ TileArgsOf<RS> sargs;    // the record of the current tile
    __shared__ int smode;
    const int tid = threadIdx.x;
    const long long K = __ldcg(p.kstep);
    const int ntiles = p.ntiles;

    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0: resolve the tile's slot and origin, remember them for the stage, load it
    auto issue = [&](int tile, int s) {
        const int a = find_owner(p.tile_begin, p.nactive, tile);
        const int slot = __ldg(&p.active[a]);
        const int rel = tile - __ldg(&p.tile_begin[a]);
        const SlotDesc* d = p.desc + slot;
        const int ntx = __ldg(&d->ntx);
        const int ty = rel / ntx;
        const int x0 = (rel - ty * ntx) * TX, y0 = ty * TY;
        const long long sl = K - __ldg(&d->k_start);
        const CUtensorMap* map = p.maps + 2 * slot + (int)(sl & 1);
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
        st_slot[s] = slot;
        st_x0[s] = x0;
        st_y0[s] = y0;
        const int gx = __ldg(&d->g.gx);
        const uint32_t bar = smem_u32(&mbar[s]);
        mbar_expect_tx(bar, TT::TX_BYTES);
        float* st = smem + s * TT::STAGE;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            tma_load_3d(smem_u32(st + i * TT::PS), map, x0 - TT::XO + gx, y0 - 1 - kCYt[i] + GY, i, bar);
    };

    const int first = blockIdx.x;
    if (tid == 0) {
        if (first < ntiles) issue(first, 0);
        if (first + (int)gridDim.x < ntiles) issue(first + gridDim.x, 1);
    }
    __syncthreads();   // the slots and origins of the first two tiles are visible to all
    int k = 0;
    for (int tile = first; tile < ntiles; tile += gridDim.x, ++k) {
        const int s = k & 1;
        // the tile's slot and origin (written before the previous barrier) are read while
        // its populations are in flight
        const int slot = st_slot[s], x0 = st_x0[s], y0 = st_y0[s];
        const SlotDesc* d = p.desc + slot;
        const long long sl = K - __ldg(&d->k_start);
        const bool ok = mbar_wait_bounded(smem_u32(&mbar[s]), (uint32_t)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(p.err, 1);
                mbar_wait_bounded(smem_u32(&mbar[s]), (uint32_t)((k >> 1) & 1));
                if (tile + (int)gridDim.x < ntiles)
                    mbar_wait_bounded(smem_u32(&mbar[s ^ 1]), (uint32_t)(((k + 1) >> 1) & 1));
            }
            break;
        }
        Grid g;
        g.nx = __ldg(&d->g.nx); g.ny = __ldg(&d->g.ny); g.gx = __ldg(&d->g.gx);
        g.pitch = __ldg(&d->g.pitch); g.plane = __ldg(&d->g.plane);
        float* dst = (sl & 1) ? d->buf[0] : d->buf[1];
        const float* S = smem + s * TT::STAGE;
        // the slot's record, to shared memory (its last readers, the previous tile's
        // collision, are past the barrier above)
        if (tid == 0) {
            load_tile_args(p.recs + slot, sl, &sargs, &smode);
            if constexpr (RS) {
                if (smode == 3) load_stencil_args(p.recs + slot, &sargs);
            }
        }

        // pulled populations stay in registers across the density barrier; the stage is
        // refilled right after it (slot, x0, y0 are in registers by then)
        float fr[TX * TY / NT][Q];
        tile_pull<TX, TY, NT, RS>(S, R, fr);
        __syncthreads();
        const int mode = smode;
        if (tid == 0 && !(RS && mode == 3) && tile + 2 * (int)gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tile + 2 * gridDim.x, s);
        }
        bool stepped = false;
        if constexpr (RS) {
            if (mode == 3) {
                // real-space correlated noise: contributions in the consumed stage s, refilled
                // after the collision (the mode is the tile's: uniform over the CTA)
                float2* Hs = reinterpret_cast<float2*>(smem_raw + s * TT::STAGE_BYTES);
                tile_stencil<TX, TY, NT>(sargs, Hs, g, x0, y0);
                __syncthreads();
                tile_nodes<3, TX, TY, NT>(sargs, fr, R, g, x0, y0, dst, nullptr, Hs);
                __syncthreads();
                if (tid == 0 && tile + 2 * (int)gridDim.x < ntiles) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(tile + 2 * gridDim.x, s);
                }
                stepped = true;
            }
        }
        if (!stepped) {
            if (mode == 2) tile_nodes<2, TX, TY, NT>(sargs, fr, R, g, x0, y0, dst, d->xi);
            else if (mode) tile_nodes<1, TX, TY, NT>(sargs, fr, R, g, x0, y0, dst, nullptr);
            else tile_nodes<0, TX, TY, NT>(sargs, fr, R, g, x0, y0, dst, nullptr);
        }
    }
    if (tid == 0) {
        const unsigned int prev = atomicAdd(p.done, 1u);
        if (prev == gridDim.x - 1) {
            *p.done = 0u;
            *p.kstep = K + 1;
        }
    }
}

// Correlated noise of the served simulations of one size: k-space synthesis with each
// simulation's Xi(k) coefficients, seed and own time, back along y (blockIdx.y = the
// simulation's index in `slots`), then back along x (one CTA per row).
__global__ void __launch_bounds__(1024) serve_noise_cols_kernel(const int* __restrict__ slots,
                                                                const SlotDesc* __restrict__ desc,
                                                                const RepRec* __restrict__ recs,
                                                                const long long* __restrict__ kstep, int nx, int ny,
                                                                int count, const float2* __restrict__ twy,
                                                                const float* __restrict__ cosx,
                                                                const float* __restrict__ cosy) {
    const int slot = __ldg(&slots[blockIdx.y]);
    const RepRec* rp = recs + slot;
    NoiseGenT<KeyPair> ga;
    ga.a44 = __ldg(&rp->a44); ga.b44 = __ldg(&rp->b44);
    ga.a49 = __ldg(&rp->a49); ga.b49 = __ldg(&rp->b49);
    ga.a99 = __ldg(&rp->a99); ga.b99 = __ldg(&rp->b99);
    ga.eig = 0;
    ga.cosx = cosx; ga.cosy = cosy;
    ga.nx = nx; ga.ny = ny;
    const long long t = __ldcg(kstep) - __ldg(&desc[slot].k_start);
    ga.t_lo = (uint32_t)((unsigned long long)t & 0xffffffffu);
    ga.t_hi = (uint32_t)((unsigned long long)t >> 32);
    ga.rk.k0 = __ldg(&rp->k0);
    ga.rk.k1 = __ldg(&rp->k1);
    noise_cols_block<false>(desc[slot].xi, ga, count, blockIdx.x, twy);
}

__global__ void __launch_bounds__(1024) serve_noise_rows_kernel(const int* __restrict__ slots,
                                                                const SlotDesc* __restrict__ desc, int nx, int ny,
                                                                const float2* __restrict__ twx, float scale) {
    extern __shared__ float2 sm[];
    const int slot = __ldg(&slots[blockIdx.x / ny]);
    float2* rowp = desc[slot].xi + (long long)(blockIdx.x % ny) * nx;
    if (nx >= 256) {
        stockham_fft_io(sm, nx, 31 - __clz(nx), 1, -1, twx, [&](int e) { return rowp[e]; },
                        [&](int e, float2 v) { rowp[e] = make_float2(v.x * scale, v.y * scale); });
        return;
    }
    for (int j = threadIdx.x; j < nx; j += blockDim.x) sm[fpad(j)] = rowp[j];
    stockham_fft(sm, nx, 31 - __clz(nx), 1, -1, twx);
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        const float2 v = sm[fpad(j)];
        rowp[j] = make_float2(v.x * scale, v.y * scale);
    }
}

static bool make_slot_map(void* buf, const Grid& g, CUtensorMap* map) {
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * GY), (cuuint64_t)Q};
    cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4};
    cuuint32_t box[3] = {(cuuint32_t)(SV_TX + 8), (cuuint32_t)(SV_TY + 2), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    // 64-byte L2 promotion, as for the batched engine's class maps (lb_batch.cu): the slot's
    // ghost columns are mostly never read
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbf

using namespace lbf;

namespace {

constexpr double SIGMA_S2_S = 1.0 / 3.0;

using Clock = std::chrono::steady_clock;

size_t align256s(size_t v) { return (v + 255) & ~size_t(255); }

bool serve_grid(int nx, int ny, Grid* g) {
    if (nx < 2 || ny < 2 || nx > 16384 || ny > 16384) return false;
    g->nx = nx; g->ny = ny; g->gx = 32;
    g->pitch = (nx + 64 + 31) / 32 * 32;
    g->plane = ((long long)g->pitch * (ny + 2 * GY) + 63) / 64 * 64;
    return true;
}

// device memory of one request: two population buffers, then (correlated noise only) its
// (xi_4, xi_9) field
size_t buf_bytes(const Grid& g) { return align256s((size_t)Q * g.plane * sizeof(float)); }
size_t slot_bytes(const Grid& g, bool full = false) {
    return 2 * buf_bytes(g) + (full ? align256s((size_t)g.nx * g.ny * sizeof(float2)) : 0);
}

bool pow2s(int v) { return v >= 2 && (v & (v - 1)) == 0; }

// k-space column strip of the correlated-noise synthesis (as the single-lattice path)
int noise_strip(int nx, int ny) {
    int c = 16;
    while (c > 1 && (fft_threads(ny, c) > 1024 || fft_smem_bytes(ny, c) > 200 * 1024)) c >>= 1;
    return c > nx ? nx : c;
}

struct Pending {
    lb_request r;                                  // r.init is null: the state is in `init`
    std::shared_ptr<std::vector<double>> init;     // initial populations (host copy), or null
    int64_t id;
    double t_submit;
};

struct Running {
    lb_request r;
    int64_t id;
    int slot;
    Grid g;
    char* mem;
    size_t bytes;
    long long k_start, k_end;
    double t_submit, t_admit;
    bool finished = false;       // its last step has been issued
    int chunk = -1;              // chunk that issues its last step
    bool full = false;           // correlated noise (needs the k-space synthesis every step)
};

struct Kept {
    Running run;
};

}  // namespace

struct SizeTables {                  // FFT twiddles and cosines of one lattice size
    float2* twx = nullptr;
    float2* twy = nullptr;
    float* cosx = nullptr;
    float* cosy = nullptr;
};

struct lb_server {
    int device = 0;
    size_t budget = 0, in_use = 0, peak = 0;
    int max_slots = 0, max_chunk = 0, grid = 0, grid_rs = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    // device tables
    CUtensorMap* d_maps = nullptr;
    SlotDesc* d_desc = nullptr;
    RepRec* d_recs = nullptr;
    double* d_fbar = nullptr;        // [slot][9]
    double* d_sums = nullptr;        // [slot][3]
    int* d_active[2] = {nullptr, nullptr};
    int* d_full[2] = {nullptr, nullptr};     // correlated simulations of a chunk, grouped by size
    int* h_full[2] = {nullptr, nullptr};
    std::map<std::pair<int, int>, SizeTables> tables;
    size_t noise_csm = 0, noise_rsm = 0;     // shared memory the noise kernels are set up for
    int* d_tb[2] = {nullptr, nullptr};
    long long* d_k = nullptr;
    unsigned int* d_done = nullptr;
    int* d_err = nullptr;
    double* d_partial = nullptr;
    // pinned host staging
    int* h_active[2] = {nullptr, nullptr};
    int* h_tb[2] = {nullptr, nullptr};
    double* h_sums = nullptr;        // [slot][3]
    int* h_err = nullptr;            // [2]: error word after the chunk of that parity
    unsigned char* h_slot = nullptr; // per slot: 2 maps, desc, record, fbar
    size_t slot_stage = 0;
    // scheduling state (worker thread)
    std::vector<int> free_slots;
    std::vector<Running> running;
    long long K = 0;
    int chunk_id = 0;
    cudaEvent_t ev_begin[2] = {nullptr, nullptr}, ev_end[2] = {nullptr, nullptr};
    std::vector<Running> in_flight[2];  // finished in the chunk of that parity
    bool chunk_pending[2] = {false, false};
    // shared with the API threads
    std::mutex mu;
    std::mutex gpu;                   // held while issuing GPU work on `stream`
    std::condition_variable cv, cv_done;
    std::deque<Pending> queue;
    std::vector<lb_result> results;   // completed, not yet polled
    std::unordered_map<int64_t, lb_result> all_results;
    std::unordered_map<int64_t, Kept> kept;
    int64_t next_id = 1;
    long long submitted = 0, completed = 0;
    double node_updates = 0.0, busy_ms = 0.0;
    double t_first_admit = -1.0, t_last_complete = -1.0;
    bool stop = false;
    int inject_alloc_fail = 0;        // host-side fault injection: admissions left to fail
    long long large_nodes = 0;        // admission: requests with at least this many nodes ...
    int max_large = 0;                // ... are admitted at most this many at a time (0: no limit)
    std::vector<int64_t> cancel_ids;  // admitted requests to withdraw at the next chunk boundary
    std::string err;                  // sticky worker error
    std::thread worker;
    Clock::time_point t0;
};

namespace {

double now_s(const lb_server* s) { return std::chrono::duration<double>(Clock::now() - s->t0).count(); }

unsigned char* slot_stage(lb_server* s, int slot) { return s->h_slot + (size_t)slot * s->slot_stage; }

// worker-side CUDA check: records a sticky error and stops the worker
#define SCK(s, call)                                                                 \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            std::lock_guard<std::mutex> lk_((s)->mu);                                \
            (s)->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return false;                                                            \
        }                                                                            \
    } while (0)

// twiddles and cosines of a lattice size for the correlated noise (first request of the size)
bool ensure_tables(lb_server* s, int nx, int ny) {
    auto key = std::make_pair(nx, ny);
    if (s->tables.count(key)) return true;
    SizeTables t;
    SCK(s, cudaMalloc(&t.twx, nx * sizeof(float2)));
    SCK(s, cudaMalloc(&t.twy, ny * sizeof(float2)));
    SCK(s, cudaMalloc(&t.cosx, nx * sizeof(float)));
    SCK(s, cudaMalloc(&t.cosy, ny * sizeof(float)));
    for (int which = 0; which < 2; ++which) {
        const int n = which == 0 ? nx : ny;
        std::vector<float2> tw(n);
        std::vector<float> cs(n);
        for (int k = 0; k < n; ++k) {
            const double a = 2.0 * M_PI * (double)k / n;
            tw[k] = make_float2((float)std::cos(a), (float)-std::sin(a));
            cs[k] = (float)std::cos(a);
        }
        SCK(s, cudaMemcpy(which == 0 ? t.twx : t.twy, tw.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
        SCK(s, cudaMemcpy(which == 0 ? t.cosx : t.cosy, cs.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    s->tables[key] = t;
    const size_t csm = fft_smem_bytes(ny, noise_strip(nx, ny)), rsm = fft_smem_bytes(nx, 1);
    if (csm > s->noise_csm) {
        SCK(s, cudaFuncSetAttribute(serve_noise_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
        s->noise_csm = csm;
    }
    if (rsm > s->noise_rsm) {
        SCK(s, cudaFuncSetAttribute(serve_noise_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
        s->noise_rsm = rsm;
    }
    return true;
}

lb_result make_result(const lb_request& r, int64_t id, int status, double t_submit, double t_admit, double t_done) {
    lb_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = id;
    res.status = status;
    res.nx = r.nx;
    res.ny = r.ny;
    res.steps = r.steps;
    res.t_submit = t_submit;
    res.t_admit = t_admit;
    res.t_complete = t_done;
    return res;
}

// a request that leaves without (further) running: its budget and slot are returned
void finish_unrun(lb_server* s, const Running& run, int status) {
    const double t = now_s(s);
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use -= run.bytes;
    s->free_slots.push_back(run.slot);
    lb_result res = make_result(run.r, run.id, status, run.t_submit, t, t);
    s->results.push_back(res);
    s->all_results[run.id] = res;
    s->completed++;
    s->cv_done.notify_all();
}

// withdraw the admitted requests whose cancellation was asked for
bool apply_cancellations(lb_server* s) {
    std::vector<int64_t> ids;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        ids.swap(s->cancel_ids);
    }
    for (int64_t id : ids) {
        for (auto it = s->running.begin(); it != s->running.end(); ++it) {
            if (it->id != id) continue;
            {
                // the slot's staging copies and the chunks in flight must be done before
                // the slot can be handed to another request (a rare path: synchronise)
                std::lock_guard<std::mutex> gl(s->gpu);
                SCK(s, cudaFreeAsync(it->mem, s->stream));
                SCK(s, cudaStreamSynchronize(s->stream));
            }
            finish_unrun(s, *it, LB_ECANCELED);
            s->running.erase(it);
            break;
        }
    }
    return true;
}

// admit pending requests (arrival order, smaller ones may pass a request that does not fit)
bool admit(lb_server* s) {
    std::vector<Pending> take;
    std::vector<int> slots;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // large requests already admitted (the admission limit on them, if set)
        int large = 0;
        if (s->max_large > 0)
            for (const Running& r : s->running) large += (long long)r.g.nx * r.g.ny >= s->large_nodes;
        for (auto it = s->queue.begin(); it != s->queue.end() && !s->free_slots.empty();) {
            Grid g;
            serve_grid(it->r.nx, it->r.ny, &g);
            const size_t b = slot_bytes(g, it->r.noise_mode == LB_NOISE_FULL);
            const bool is_large = s->max_large > 0 && (long long)it->r.nx * it->r.ny >= s->large_nodes;
            if (is_large && large >= s->max_large) {
                ++it;                  // waits for a large one to finish; smaller ones may pass
                continue;
            }
            if (s->in_use + b <= s->budget) {
                large += is_large;
                s->in_use += b;
                s->peak = std::max(s->peak, s->in_use);
                take.push_back(*it);
                slots.push_back(s->free_slots.back());
                s->free_slots.pop_back();
                it = s->queue.erase(it);
            } else {
                ++it;
            }
        }
    }
    if (take.empty()) return true;
    std::lock_guard<std::mutex> gl(s->gpu);
    for (size_t q = 0; q < take.size(); ++q) {
        const Pending& pr = take[q];
        Running run;
        run.r = pr.r;
        run.id = pr.id;
        run.t_submit = pr.t_submit;
        serve_grid(pr.r.nx, pr.r.ny, &run.g);
        run.full = pr.r.noise_mode == LB_NOISE_FULL && pr.r.kT > 0.0;
        run.bytes = slot_bytes(run.g, pr.r.noise_mode == LB_NOISE_FULL);
        run.slot = slots[q];
        bool injected = false;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->inject_alloc_fail > 0) {
                s->inject_alloc_fail--;
                injected = true;
            }
        }
        // an injected failure takes the same path as a real one: the request completes
        // with LB_ENOMEM, unrun, and the server carries on
        void* mem = nullptr;
        cudaError_t ae = injected ? cudaErrorMemoryAllocation
                                  : cudaMallocFromPoolAsync(&mem, run.bytes, s->pool, s->stream);
        if (ae == cudaErrorMemoryAllocation) {
            cudaGetLastError();            // not sticky: clear it
            finish_unrun(s, run, LB_ENOMEM);
            continue;
        }
        SCK(s, ae);
        run.mem = (char*)mem;
        SCK(s, cudaMemsetAsync(run.mem, 0, run.bytes, s->stream));   // rest: zero deviations
        if (pr.init) {
            // the caller's initial state, through an FP64 staging plane taken from the pool
            // for the upload only
            const long long n = (long long)run.g.nx * run.g.ny;
            void* stage = nullptr;
            ae = cudaMallocFromPoolAsync(&stage, (size_t)n * sizeof(double), s->pool, s->stream);
            if (ae == cudaErrorMemoryAllocation) {
                cudaGetLastError();
                SCK(s, cudaFreeAsync(run.mem, s->stream));
                finish_unrun(s, run, LB_ENOMEM);
                continue;
            }
            SCK(s, ae);
            double fb0[Q];
            rest_populations(pr.r.rho0, pr.r.cs2, fb0);
            for (int i = 0; i < Q; ++i) {
                SCK(s, cudaMemcpyAsync(stage, pr.init->data() + (size_t)i * n, (size_t)n * sizeof(double),
                                       cudaMemcpyHostToDevice, s->stream));
                SCK(s, launch_set_plane((const double*)stage, run.mem, 0, run.g, i, fb0[i], s->stream));
            }
            SCK(s, cudaFreeAsync(stage, s->stream));
        }
        float* b0 = reinterpret_cast<float*>(run.mem);
        float* b1 = reinterpret_cast<float*>(run.mem + buf_bytes(run.g));
        unsigned char* st = slot_stage(s, run.slot);
        CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(st);
        if (!make_slot_map(b0, run.g, &maps[0]) || !make_slot_map(b1, run.g, &maps[1])) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->err = "cuTensorMapEncodeTiled failed";
            return false;
        }
        SlotDesc* d = reinterpret_cast<SlotDesc*>(st + 2 * sizeof(CUtensorMap));
        d->g = run.g;
        d->buf[0] = b0;
        d->buf[1] = b1;
        d->xi = nullptr;
        if (run.full) {
            d->xi = reinterpret_cast<float2*>(run.mem + 2 * buf_bytes(run.g));
            if (!ensure_tables(s, run.g.nx, run.g.ny)) return false;
        }
        d->ntx = (run.g.nx + SV_TX - 1) / SV_TX;
        d->k_start = s->K;
        RepRec* rec = reinterpret_cast<RepRec*>(st + 2 * sizeof(CUtensorMap) + sizeof(SlotDesc));
        std::memset(rec, 0, sizeof(RepRec));
        rec->rho0 = (float)pr.r.rho0;
        rec->cs2m = (float)(pr.r.cs2 - SIGMA_S2_S);
        fill_rep_record(pr.r.rho0, pr.r.cs2, pr.r.kT, pr.r.kappa, pr.r.tau_s, pr.r.tau_b, pr.r.tau_ghost,
                        pr.r.noise_mode, rec);
        rec->k0 = (uint32_t)(pr.r.seed & 0xffffffffu);
        rec->k1 = (uint32_t)(pr.r.seed >> 32);
        rec->toff = 0;
        double* fb = reinterpret_cast<double*>(st + 2 * sizeof(CUtensorMap) + sizeof(SlotDesc) + sizeof(RepRec));
        rest_populations(pr.r.rho0, pr.r.cs2, fb);
        SCK(s, cudaMemcpyAsync(s->d_maps + 2 * run.slot, maps, 2 * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                               s->stream));
        SCK(s, cudaMemcpyAsync(s->d_desc + run.slot, d, sizeof(SlotDesc), cudaMemcpyHostToDevice, s->stream));
        SCK(s, cudaMemcpyAsync(s->d_recs + run.slot, rec, sizeof(RepRec), cudaMemcpyHostToDevice, s->stream));
        SCK(s, cudaMemcpyAsync(s->d_fbar + (size_t)Q * run.slot, fb, Q * sizeof(double), cudaMemcpyHostToDevice,
                               s->stream));
        run.k_start = s->K;
        run.k_end = s->K + pr.r.steps;
        run.t_admit = now_s(s);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->t_first_admit < 0) s->t_first_admit = run.t_admit;
        }
        s->running.push_back(run);
    }
    return true;
}

// results of the simulations whose last step was in the chunk of parity c, after its event
bool complete_chunk(lb_server* s, int c) {
    if (!s->chunk_pending[c]) return true;
    SCK(s, cudaEventSynchronize(s->ev_end[c]));
    float ms = 0.f;
    SCK(s, cudaEventElapsedTime(&ms, s->ev_begin[c], s->ev_end[c]));
    const int hflag = s->h_err[c];
    const double t = now_s(s);
    std::lock_guard<std::mutex> lk(s->mu);
    s->busy_ms += ms;
    if (hflag) s->err = "a served step kernel gave up waiting for its TMA loads";
    for (Running& run : s->in_flight[c]) {
        lb_result res;
        std::memset(&res, 0, sizeof(res));
        res.id = run.id;
        res.status = hflag ? LB_ETIMEOUT : LB_OK;
        res.nx = run.r.nx;
        res.ny = run.r.ny;
        res.steps = run.r.steps;
        for (int j = 0; j < 3; ++j) res.sums[j] = s->h_sums[3 * run.slot + j];
        if (res.status == LB_OK && !(std::isfinite(res.sums[0]) && std::isfinite(res.sums[1]) &&
                                     std::isfinite(res.sums[2])))
            res.status = LB_ENONFINITE;
        res.t_submit = run.t_submit;
        res.t_admit = run.t_admit;
        res.t_complete = t;
        res.state_kept = run.r.keep_state ? 1 : 0;
        s->results.push_back(res);
        s->all_results[run.id] = res;
        s->completed++;
        s->t_last_complete = t;
        if (run.r.keep_state) {
            s->kept[run.id] = Kept{run};
        } else {
            s->free_slots.push_back(run.slot);
        }
    }
    s->in_flight[c].clear();
    s->chunk_pending[c] = false;
    s->cv_done.notify_all();
    return true;
}

// one chunk: steps for every running simulation up to the earliest end (capped)
bool issue_chunk(lb_server* s) {
    if (s->running.empty()) return true;
    const int c = s->chunk_id & 1;
    // the staging of parity c was last used two chunks ago: wait for that chunk first
    if (!complete_chunk(s, c)) return false;
    long long G = s->max_chunk;
    for (const Running& r : s->running) G = std::min(G, r.k_end - s->K);
    int* act = s->h_active[c];
    int* tb = s->h_tb[c];
    int tiles = 0;
    double nodes = 0.0;
    for (size_t a = 0; a < s->running.size(); ++a) {
        const Running& r = s->running[a];
        act[a] = r.slot;
        tb[a] = tiles;
        tiles += ((r.g.nx + SV_TX - 1) / SV_TX) * ((r.g.ny + SV_TY - 1) / SV_TY);
        nodes += (double)r.g.nx * r.g.ny;
    }
    const int n = (int)s->running.size();
    tb[n] = tiles;
    // correlated simulations grouped by size: one pair of noise launches per size and step
    struct Group { int nx, ny, off, cnt; };
    std::vector<Group> groups;
    {
        std::map<std::pair<int, int>, std::vector<int>> by;
        for (const Running& r : s->running)
            if (r.full) by[std::make_pair(r.g.nx, r.g.ny)].push_back(r.slot);
        int off = 0;
        for (auto& kv : by) {
            for (size_t q = 0; q < kv.second.size(); ++q) s->h_full[c][off + q] = kv.second[q];
            groups.push_back(Group{kv.first.first, kv.first.second, off, (int)kv.second.size()});
            off += (int)kv.second.size();
        }
    }
    std::lock_guard<std::mutex> gl(s->gpu);
    SCK(s, cudaMemcpyAsync(s->d_active[c], act, n * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    SCK(s, cudaMemcpyAsync(s->d_tb[c], tb, (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    if (!groups.empty()) {
        const int nf = groups.back().off + groups.back().cnt;
        SCK(s, cudaMemcpyAsync(s->d_full[c], s->h_full[c], nf * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    }
    ServeParams p;
    p.maps = s->d_maps;
    p.desc = s->d_desc;
    p.recs = s->d_recs;
    p.active = s->d_active[c];
    p.tile_begin = s->d_tb[c];
    p.nactive = n;
    p.ntiles = tiles;
    p.kstep = s->d_k;
    p.done = s->d_done;
    p.err = s->d_err;
    using TT = TmaTile<SV_TX, SV_TY, float>;
    bool rs = false;
    for (const Running& r : s->running) rs = rs || (r.r.noise_mode == LB_NOISE_FULL_RS && r.r.kT > 0.0);
    const int grid = std::max(1, std::min(tiles, rs ? s->grid_rs : s->grid));
    SCK(s, cudaEventRecord(s->ev_begin[c], s->stream));
    for (long long k = 0; k < G; ++k) {
        for (const Group& gr : groups) {
            const SizeTables& tb2 = s->tables[std::make_pair(gr.nx, gr.ny)];
            const int cs = noise_strip(gr.nx, gr.ny);
            serve_noise_cols_kernel<<<dim3(gr.nx / cs, gr.cnt), fft_threads(gr.ny, cs), fft_smem_bytes(gr.ny, cs),
                                      s->stream>>>(s->d_full[c] + gr.off, s->d_desc, s->d_recs, s->d_k, gr.nx, gr.ny,
                                                   cs, tb2.twy, tb2.cosx, tb2.cosy);
            serve_noise_rows_kernel<<<gr.cnt * gr.ny, fft_threads(gr.nx, 1), fft_smem_bytes(gr.nx, 1), s->stream>>>(
                s->d_full[c] + gr.off, s->d_desc, gr.nx, gr.ny, tb2.twx,
                (float)(1.0 / std::sqrt((double)gr.nx * gr.ny)));
        }
        if (rs) step_serve_kernel<SV_TX, SV_TY, SV_NT, true><<<grid, SV_NT, TT::SMEM_BYTES, s->stream>>>(p);
        else step_serve_kernel<SV_TX, SV_TY, SV_NT, false><<<grid, SV_NT, TT::SMEM_BYTES, s->stream>>>(p);
    }
    SCK(s, cudaGetLastError());
    s->K += G;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->node_updates += nodes * (double)G;
    }
    // simulations that end here: conserved sums of their final state, then release
    for (auto it = s->running.begin(); it != s->running.end();) {
        if (it->k_end != s->K) { ++it; continue; }
        const int fin = (int)(it->r.steps & 1);   // buffer holding the state after `steps` steps
        float* pops = reinterpret_cast<float*>(it->mem + (fin ? buf_bytes(it->g) : 0));
        SCK(s, launch_sums(pops, 0, it->g, s->d_fbar + (size_t)Q * it->slot, s->d_partial, s->d_sums + 3 * it->slot,
                           s->stream));
        SCK(s, cudaMemcpyAsync(s->h_sums + 3 * it->slot, s->d_sums + 3 * it->slot, 3 * sizeof(double),
                               cudaMemcpyDeviceToHost, s->stream));
        if (!it->r.keep_state) {
            SCK(s, cudaFreeAsync(it->mem, s->stream));
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= it->bytes;
        }
        s->in_flight[c].push_back(*it);
        it = s->running.erase(it);
    }
    SCK(s, cudaMemcpyAsync(s->h_err + c, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaEventRecord(s->ev_end[c], s->stream));
    s->chunk_pending[c] = true;
    s->chunk_id++;
    return true;
}

void worker_main(lb_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (!s->err.empty()) break;
            const bool idle = s->running.empty() && !s->chunk_pending[0] && !s->chunk_pending[1];
            if (idle && s->queue.empty()) {
                s->cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            }
            if (s->stop && s->queue.empty() && s->running.empty() && !s->chunk_pending[0] && !s->chunk_pending[1])
                break;
        }
        if (!apply_cancellations(s)) break;
        if (!admit(s)) break;
        if (s->running.empty()) {
            // nothing admitted (budget or slots held by chunks in flight): finish those first
            if (!complete_chunk(s, (s->chunk_id + 1) & 1)) break;
            if (!complete_chunk(s, s->chunk_id & 1)) break;
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->running.empty() && !s->queue.empty() && s->free_slots.size() > 0) {
                // a request that cannot be admitted yet waits for kept states to be released
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
            }
            continue;
        }
        if (!issue_chunk(s)) break;
    }
    // drain whatever is still in flight
    complete_chunk(s, 0);
    complete_chunk(s, 1);
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_done.notify_all();
}

int sfail(lb_server* s, int code, const std::string& m) {
    if (s) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = s->err.empty() ? m : s->err;
    } else {
        set_context_free_error(m);
    }
    return code;
}

}  // namespace

extern "C" {

size_t lb_server_request_bytes(int nx, int ny, int noise_mode) {
    Grid g;
    if (!serve_grid(nx, ny, &g)) return 0;
    return slot_bytes(g, noise_mode == LB_NOISE_FULL);
}

int lb_server_create(size_t hbm_budget_bytes, int max_active, int max_chunk_steps, lb_server** out) {
    if (!out || hbm_budget_bytes == 0 || max_active < 1 || max_active > (1 << 16) || max_chunk_steps < 1)
        return sfail(nullptr, LB_EINVAL, "invalid server limits");
    *out = nullptr;
    lb_server* s = new lb_server();
    s->budget = hbm_budget_bytes;
    s->max_slots = max_active;
    s->max_chunk = max_chunk_steps;
    s->t0 = Clock::now();
    cudaGetDevice(&s->device);
    s->slot_stage = align256s(2 * sizeof(CUtensorMap) + sizeof(SlotDesc) + sizeof(RepRec) + Q * sizeof(double));
    auto fail_create = [&](cudaError_t e) {
        set_context_free_error(std::string("lb_server_create: ") + cudaGetErrorString(e));
        lb_server_destroy(s);
        return LB_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) return fail_create(e);
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if ((e = cudaMemPoolCreate(&s->pool, &props)) != cudaSuccess) return fail_create(e);
    cuuint64_t keep = hbm_budget_bytes;           // freed blocks stay in the pool up to the budget
    if ((e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
        return fail_create(e);
    const size_t M = (size_t)max_active;
    if ((e = cudaMalloc(&s->d_maps, M * 2 * sizeof(CUtensorMap))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMalloc(&s->d_desc, M * sizeof(SlotDesc))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMalloc(&s->d_recs, M * sizeof(RepRec))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMalloc(&s->d_fbar, M * Q * sizeof(double))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMalloc(&s->d_sums, M * 3 * sizeof(double))) != cudaSuccess) return fail_create(e);
    for (int c = 0; c < 2; ++c) {
        if ((e = cudaMalloc(&s->d_active[c], M * sizeof(int))) != cudaSuccess) return fail_create(e);
        if ((e = cudaMalloc(&s->d_tb[c], (M + 1) * sizeof(int))) != cudaSuccess) return fail_create(e);
        if ((e = cudaMallocHost(&s->h_active[c], M * sizeof(int))) != cudaSuccess) return fail_create(e);
        if ((e = cudaMallocHost(&s->h_tb[c], (M + 1) * sizeof(int))) != cudaSuccess) return fail_create(e);
        if ((e = cudaMalloc(&s->d_full[c], M * sizeof(int))) != cudaSuccess) return fail_create(e);
        if ((e = cudaMallocHost(&s->h_full[c], M * sizeof(int))) != cudaSuccess) return fail_create(e);
        if ((e = cudaEventCreate(&s->ev_begin[c])) != cudaSuccess) return fail_create(e);
        if ((e = cudaEventCreate(&s->ev_end[c])) != cudaSuccess) return fail_create(e);
    }
    if ((e = cudaMalloc(&s->d_k, sizeof(long long))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMalloc(&s->d_done, sizeof(unsigned int))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMalloc(&s->d_err, sizeof(int))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMalloc(&s->d_partial, (size_t)sums_partial_count() * sizeof(double))) != cudaSuccess)
        return fail_create(e);
    if ((e = cudaMallocHost(&s->h_sums, M * 3 * sizeof(double))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMallocHost(&s->h_err, 2 * sizeof(int))) != cudaSuccess) return fail_create(e);
    s->h_err[0] = s->h_err[1] = 0;
    if ((e = cudaMallocHost(&s->h_slot, M * s->slot_stage)) != cudaSuccess) return fail_create(e);
    if ((e = cudaMemset(s->d_k, 0, sizeof(long long))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMemset(s->d_done, 0, sizeof(unsigned int))) != cudaSuccess) return fail_create(e);
    if ((e = cudaMemset(s->d_err, 0, sizeof(int))) != cudaSuccess) return fail_create(e);
    using TT = TmaTile<SV_TX, SV_TY, float>;
    auto kern = step_serve_kernel<SV_TX, SV_TY, SV_NT, false>;
    auto kern_rs = step_serve_kernel<SV_TX, SV_TY, SV_NT, true>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TT::SMEM_BYTES)) != cudaSuccess)
        return fail_create(e);
    if ((e = cudaFuncSetAttribute(kern_rs, cudaFuncAttributeMaxDynamicSharedMemorySize, TT::SMEM_BYTES)) !=
        cudaSuccess)
        return fail_create(e);
    int sms = 0, per = 0, per_rs = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, SV_NT, TT::SMEM_BYTES)) != cudaSuccess)
        return fail_create(e);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_rs, kern_rs, SV_NT, TT::SMEM_BYTES)) != cudaSuccess)
        return fail_create(e);
    s->grid = sms * std::max(per, 1);
    s->grid_rs = sms * std::max(per_rs, 1);
    if (!tensor_map_encoder()) {
        set_context_free_error("lb_server_create: cuTensorMapEncodeTiled is not available");
        lb_server_destroy(s);
        return LB_ECUDA;
    }
    for (int i = max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return LB_OK;
}

int lb_server_submit(lb_server* s, const lb_request* r, int64_t* id) {
    if (!s || !r) return LB_EINVAL;
    Grid g;
    if (!serve_grid(r->nx, r->ny, &g)) return sfail(nullptr, LB_EINVAL, "lattice sides must lie in [2, 16384]");
    if (r->steps < 1) return sfail(nullptr, LB_EINVAL, "steps must be >= 1");
    if (r->noise_mode == LB_NOISE_FULL &&
        (!pow2s(r->nx) || !pow2s(r->ny) || r->ny > 8192 || noise_strip(r->nx, r->ny) < 2))
        return sfail(nullptr, LB_EINVAL, "correlated noise needs nx and ny powers of two and ny <= 8192");
    if (r->noise_mode == LB_NOISE_LW_LOCAL)
        return sfail(nullptr, LB_EINVAL, "served simulations use homogeneous noise modes only (not LB_NOISE_LW_LOCAL)");
    const int rc = lb_check_params(r->nx, r->ny, r->rho0, r->cs2, r->kT, r->kappa, r->tau_s, r->tau_b, r->tau_ghost,
                                   r->noise_mode);
    if (rc != LB_OK) return sfail(nullptr, rc, "parameters rejected (see lb_check_params)");
    if (slot_bytes(g, r->noise_mode == LB_NOISE_FULL) > s->budget)
        return sfail(nullptr, LB_ENOMEM, "the request alone exceeds the HBM budget");
    std::shared_ptr<std::vector<double>> init_copy;
    if (r->init) {
        const size_t cnt = (size_t)Q * r->nx * r->ny;
        init_copy = std::make_shared<std::vector<double>>(r->init, r->init + cnt);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->err.empty()) return LB_ECUDA;
    if (s->stop) return LB_ESTATE;
    Pending p;
    p.r = *r;
    p.r.init = nullptr;
    if (r->init) p.init = init_copy;
    p.id = s->next_id++;
    p.t_submit = now_s(s);
    s->queue.push_back(p);
    s->submitted++;
    if (id) *id = p.id;
    s->cv.notify_all();
    return LB_OK;
}

int lb_server_poll(lb_server* s, lb_result* out, int max_results, int* n) {
    if (!s || !n || (max_results > 0 && !out) || max_results < 0) return LB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const int k = std::min<int>(max_results, (int)s->results.size());
    for (int i = 0; i < k; ++i) out[i] = s->results[i];
    s->results.erase(s->results.begin(), s->results.begin() + k);
    *n = k;
    return s->err.empty() ? LB_OK : LB_ECUDA;
}

int lb_server_wait(lb_server* s, int64_t id, double timeout_s, lb_result* out) {
    if (!s) return LB_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                              std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
    for (;;) {
        if (!s->err.empty()) return LB_ECUDA;
        if (id > 0) {
            auto it = s->all_results.find(id);
            if (it != s->all_results.end()) {
                if (out) *out = it->second;
                return LB_OK;
            }
            if (id >= s->next_id) return LB_EINVAL;
        } else if (s->queue.empty() && s->completed == s->submitted) {
            return LB_OK;      // id <= 0: everything submitted so far has completed
        }
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return LB_ETIMEOUT;
    }
}

int lb_server_fetch_populations(lb_server* s, int64_t id, double* f) {
    if (!s || !f) return LB_EINVAL;
    Running run;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->kept.find(id);
        if (it == s->kept.end()) {
            return LB_EINVAL;     // unknown, not finished, or submitted without keep_state
        }
        run = it->second.run;
        s->kept.erase(it);
    }
    DeviceGuard dg(s->device);
    std::lock_guard<std::mutex> gl(s->gpu);
    const long long n = (long long)run.g.nx * run.g.ny;
    const int fin = (int)(run.r.steps & 1);
    const void* pops = run.mem + (fin ? buf_bytes(run.g) : 0);
    double fbar[Q];
    rest_populations(run.r.rho0, run.r.cs2, fbar);
    void* stage = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&stage, (size_t)n * sizeof(double), s->pool, s->stream);
    for (int i = 0; i < Q && e == cudaSuccess; ++i) {
        e = launch_get_plane(pops, 0, run.g, i, fbar[i], (double*)stage, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(f + i * n, stage, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    }
    if (stage) cudaFreeAsync(stage, s->stream);
    cudaFreeAsync(run.mem, s->stream);
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= run.bytes;
        s->free_slots.push_back(run.slot);
        s->cv.notify_all();
    }
    if (e != cudaSuccess || e2 != cudaSuccess)
        return sfail(s, LB_ECUDA, std::string("fetch: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return LB_OK;
}

int lb_server_get_stats(lb_server* s, lb_server_stats* st) {
    if (!s || !st) return LB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof(*st));
    st->queued = (int64_t)s->queue.size();
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->bytes_in_use = s->in_use;
    st->bytes_peak = s->peak;
    st->bytes_budget = s->budget;
    st->node_updates = s->node_updates;
    st->gpu_busy_s = s->busy_ms * 1e-3;
    st->t_first_admit = s->t_first_admit;
    st->t_last_complete = s->t_last_complete;
    st->steps_issued = s->K;
    return s->err.empty() ? LB_OK : LB_ECUDA;
}

int lb_server_cancel(lb_server* s, int64_t id) {
    if (!s) return LB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if (it->id != id) continue;
        const double t = now_s(s);
        lb_result res = make_result(it->r, id, LB_ECANCELED, it->t_submit, t, t);
        s->results.push_back(res);
        s->all_results[id] = res;
        s->completed++;
        s->queue.erase(it);
        s->cv_done.notify_all();
        return LB_OK;
    }
    if (id <= 0 || id >= s->next_id || s->all_results.count(id)) return LB_EINVAL;
    s->cancel_ids.push_back(id);      // admitted (or being admitted): withdrawn by the worker
    s->cv.notify_all();
    return LB_OK;
}

int lb_server_set_admission(lb_server* s, int64_t large_nodes, int max_large) {
    if (!s || large_nodes < 1 || max_large < 0) return LB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->large_nodes = large_nodes;
    s->max_large = max_large;
    s->cv.notify_all();
    return LB_OK;
}

int lb_server_inject_alloc_failures(lb_server* s, int count) {
    if (!s || count < 0) return LB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->inject_alloc_fail = count;
    return LB_OK;
}

int lb_server_destroy(lb_server* s) {
    if (!s) return LB_EINVAL;
    DeviceGuard dg(s->device);
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            s->queue.clear();
            s->cv.notify_all();
        }
        s->worker.join();
    }
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto& kv : s->kept) cudaFreeAsync(kv.second.run.mem, s->stream);
    for (auto& r : s->running) cudaFreeAsync(r.mem, s->stream);
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->d_maps); cudaFree(s->d_desc); cudaFree(s->d_recs); cudaFree(s->d_fbar); cudaFree(s->d_sums);
    for (int c = 0; c < 2; ++c) {
        cudaFree(s->d_active[c]); cudaFree(s->d_tb[c]);
        cudaFreeHost(s->h_active[c]); cudaFreeHost(s->h_tb[c]);
        cudaFree(s->d_full[c]); cudaFreeHost(s->h_full[c]);
        if (s->ev_begin[c]) cudaEventDestroy(s->ev_begin[c]);
        if (s->ev_end[c]) cudaEventDestroy(s->ev_end[c]);
    }
    cudaFree(s->d_k); cudaFree(s->d_done); cudaFree(s->d_err); cudaFree(s->d_partial);
    cudaFreeHost(s->h_sums); cudaFreeHost(s->h_slot); cudaFreeHost(s->h_err);
    for (auto& kv : s->tables) {
        cudaFree(kv.second.twx); cudaFree(kv.second.twy); cudaFree(kv.second.cosx); cudaFree(kv.second.cosy);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return LB_OK;
}

const char* lb_server_last_error(lb_server* s) {
    if (!s) return lb_last_error(nullptr);
    std::lock_guard<std::mutex> lk(s->mu);
    thread_local std::string copy;
    copy = s->err;
    return copy.c_str();
}

}  // extern "C"
