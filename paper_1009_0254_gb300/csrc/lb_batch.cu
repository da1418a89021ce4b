// lb_batch.cu -- many independent lattices ("replicas") stepped together.
//
// Replicas of equal size form a class.  A class keeps its populations replica-major in
// one buffer pair, [replica][plane][row][column] with the single-lattice layout per replica,
// so one 4D tensor map (x, y, plane, replica) serves the whole class.  One persistent launch
// of the batched TMA step kernel advances every replica of up to MAX_CLASSES classes by one
// step: the launch's tiles are numbered class by class, replica by replica, and every CTA
// walks its share of them through a two-stage TMA pipeline.  Each replica keeps its own
// Philox key (its seed), relaxation and noise factors and time offset in a device record;
// the step counter K lives in device memory and is advanced by the last CTA of the step's
// last launch, so a captured CUDA graph of G steps can be replayed as it is: a replica's
// time is K + offset, and K's parity selects the source buffer.  A replica stepped in a
// batch follows exactly the trajectory it would follow stepped alone.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lb_ens.cuh"
#include "lb_fft_core.cuh"
#include "lb_noise.cuh"
#include "lb_spectra.cuh"
#include "lbfluct.h"

namespace lbf {

constexpr int MAX_CLASSES = 8;      // size classes per launch (kernel parameters stay < 4 KB)

struct ClassDesc {
    Grid g;
    float* buf[2];              // the class's two population buffers
    const RepRec* recs;         // its replicas' records
    int tile_begin;             // first tile of the class in the launch's numbering
    int ntx, per;               // tiles along x per replica, tiles per replica
    unsigned long long per_m, ntx_m;   // division by per and by ntx as a multiply and a shift
    int per_s, ntx_s;
    long long rstride;          // elements per replica (9 planes)
    const float2* xi;           // correlated noise (xi_4, xi_9) of the class, nx*ny per replica, or null
};

struct EnsParams {
    CUtensorMap map[MAX_CLASSES][2];   // per class: map of buffer 0, of buffer 1
    ClassDesc cls[MAX_CLASSES];
    int nclass, ntiles;
    long long* kstep;                  // device step counter K
    unsigned int* done;                // CTAs finished in this launch (advancing launch only)
    int* err;                          // set when a bounded wait gives up
    int advance;                       // this launch advances K when its last CTA finishes
    int rs;                            // some replica of the launch has real-space correlated noise
};

// floor(n / d) for 0 <= n < 2^32 as (n m) >> s with m = ceil(2^s / d), s = 32 + ceil(log2 d)
// (Granlund and Montgomery, division by invariant integers using multiplication, 1994):
// every thread locates every tile, and a division per tile and thread is felt in the step
__device__ __forceinline__ int div_magic(int n, unsigned long long m, int s) {
    return (int)(((unsigned long long)(unsigned)n * m) >> s);
}

// class, replica and origin of a tile of the launch
struct TilePos {
    int c, rep, x0, y0;
};

template <int TX, int TY>
__device__ __forceinline__ TilePos locate(const EnsParams& p, int tile) {
    TilePos t;
    int c = 0;
#pragma unroll 1
    while (c + 1 < p.nclass && tile >= p.cls[c + 1].tile_begin) ++c;
    const ClassDesc& d = p.cls[c];
    const int rel = tile - d.tile_begin;
    t.c = c;
    t.rep = div_magic(rel, d.per_m, d.per_s);
    const int rem = rel - t.rep * d.per;
    const int ty = div_magic(rem, d.ntx_m, d.ntx_s);
    t.x0 = (rem - ty * d.ntx) * TX;
    t.y0 = ty * TY;
    return t;
}

// RS: the variant that also steps replicas with real-space correlated noise (its extra path
// raises the register count, so launches without such replicas use the lean variant)
template <int TX, int TY, int NT, bool RS>
__global__ void __launch_bounds__(NT, RS ? 1024 / NT : 0) step_ensemble_kernel(const __grid_constant__ EnsParams p) {
    using TT = TmaTile<TX, TY, float>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* smem = reinterpret_cast<float*>(smem_raw);
    float* R = reinterpret_cast<float*>(smem_raw + 2 * TT::STAGE_BYTES);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(R + TT::RW * TT::RH);
    __shared__ TileArgsOf<RS> sargs;    // the record of the current tile
    __shared__ int smode;
    const int tid = threadIdx.x;
    const long long K = __ldcg(p.kstep);
    const int par = (int)(K & 1);
    const int ntiles = p.ntiles;

    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int tile, int s) {
        const TilePos tp = locate<TX, TY>(p, tile);
        const CUtensorMap* map = &p.map[tp.c][par];
        const int gx = p.cls[tp.c].g.gx;
        const uint32_t bar = smem_u32(&mbar[s]);
        mbar_expect_tx(bar, TT::TX_BYTES);
        float* st = smem + s * TT::STAGE;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            tma_load_4d(smem_u32(st + i * TT::PS), map, tp.x0 - TT::XO + gx, tp.y0 - 1 - kCYt[i] + GY, i, tp.rep,
                        bar);
    };

    const int first = blockIdx.x;
    if (tid == 0) {
        if (first < ntiles) issue(first, 0);
        if (first + (int)gridDim.x < ntiles) issue(first + gridDim.x, 1);
    }
    int k = 0;
    for (int tile = first; tile < ntiles; tile += gridDim.x, ++k) {
        const int s = k & 1;
        const TilePos tp = locate<TX, TY>(p, tile);
        const bool ok = mbar_wait_bounded(smem_u32(&mbar[s]), (uint32_t)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(p.err, 1);
                // give the loads still in flight into this CTA's shared memory a bounded
                // chance to land before the CTA exits
                mbar_wait_bounded(smem_u32(&mbar[s]), (uint32_t)((k >> 1) & 1));
                if (tile + (int)gridDim.x < ntiles)
                    mbar_wait_bounded(smem_u32(&mbar[s ^ 1]), (uint32_t)(((k + 1) >> 1) & 1));
            }
            break;
        }
        const ClassDesc& d = p.cls[tp.c];
        const Grid g = d.g;
        const float* S = smem + s * TT::STAGE;
        // the tile's replica record, to shared memory (its last readers, the previous tile's
        // collision, are past the barrier above; measured faster than a copy per thread in
        // registers, which the pulled populations need, and than loading it before the wait)
        if (tid == 0) {
            const RepRec* rp = p.cls[tp.c].recs + tp.rep;
            load_tile_args(rp, K + __ldg(&rp->toff), &sargs, &smode);
            if constexpr (RS) {
                if (smode == 3) load_stencil_args(rp, &sargs);
            }
        }

        // pulled populations stay in registers across the density barrier; the stage is
        // refilled right after it
        float fr[TX * TY / NT][Q];
        tile_pull<TX, TY, NT, RS>(S, R, fr);
        __syncthreads();
        if (tid == 0 && !(RS && smode == 3) && tile + 2 * (int)gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tile + 2 * gridDim.x, s);
        }
        const int mode = smode;
        float* dst = (par ? d.buf[0] : d.buf[1]) + (long long)tp.rep * d.rstride;
        bool stepped = false;
        if constexpr (RS) {
            if (mode == 3) {
                // real-space correlated noise: the contributions go to the consumed stage s,
                // whose refill waits for the collision (the mode is the tile's: uniform over
                // the CTA)
                float2* Hs = reinterpret_cast<float2*>(smem_raw + s * TT::STAGE_BYTES);
                tile_stencil<TX, TY, NT>(sargs, Hs, g, tp.x0, tp.y0);
                __syncthreads();
                tile_nodes<3, TX, TY, NT>(sargs, fr, R, g, tp.x0, tp.y0, dst, nullptr, Hs);
                __syncthreads();
                if (tid == 0 && tile + 2 * (int)gridDim.x < ntiles) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(tile + 2 * gridDim.x, s);
                }
                stepped = true;
            }
        }
        if (!stepped) {
            if (mode == 2)
                tile_nodes<2, TX, TY, NT>(sargs, fr, R, g, tp.x0, tp.y0, dst, d.xi + (long long)tp.rep * g.nx * g.ny);
            else if (mode)
                tile_nodes<1, TX, TY, NT>(sargs, fr, R, g, tp.x0, tp.y0, dst, nullptr);
            else
                tile_nodes<0, TX, TY, NT>(sargs, fr, R, g, tp.x0, tp.y0, dst, nullptr);
        }
    }
    // Every CTA read K before arriving here; the last one to arrive advances it for the
    // next step (the next launch sees it, kernel boundaries order the accesses).
    if (tid == 0 && p.advance) {
        const unsigned int prev = atomicAdd(p.done, 1u);
        if (prev == gridDim.x - 1) {
            *p.done = 0u;
            *p.kstep = K + 1;
        }
    }
}

// --- correlated noise of a class -------------------------------------------------------

// First pass for every replica of the class in correlated mode (blockIdx.y = replica):
// k-space synthesis with the replica's Xi(k) coefficients, seed and time, back along y.
__global__ void __launch_bounds__(1024) batch_noise_cols_kernel(float2* out, const RepRec* __restrict__ recs,
                                                                const long long* __restrict__ kstep, int nx, int ny,
                                                                int count, const float2* __restrict__ twy,
                                                                const float* __restrict__ cosx,
                                                                const float* __restrict__ cosy) {
    const RepRec* rp = recs + blockIdx.y;
    if (__ldg(&rp->mode) != 2) return;
    NoiseGenT<KeyPair> ga;
    ga.a44 = __ldg(&rp->a44); ga.b44 = __ldg(&rp->b44);
    ga.a49 = __ldg(&rp->a49); ga.b49 = __ldg(&rp->b49);
    ga.a99 = __ldg(&rp->a99); ga.b99 = __ldg(&rp->b99);
    ga.eig = 0;
    ga.cosx = cosx; ga.cosy = cosy;
    ga.nx = nx; ga.ny = ny;
    const long long t = __ldcg(kstep) + __ldg(&rp->toff);
    ga.t_lo = (uint32_t)((unsigned long long)t & 0xffffffffu);
    ga.t_hi = (uint32_t)((unsigned long long)t >> 32);
    ga.rk.k0 = __ldg(&rp->k0);
    ga.rk.k1 = __ldg(&rp->k1);
    noise_cols_block<false>(out + (long long)blockIdx.y * nx * ny, ga, count, blockIdx.x, twy);
}

// Second pass: back along x (unitary scale).  Rows of 256 points and more: one CTA per row.
// Shorter rows: `rows` rows per CTA (a power of two dividing ny, so all of one replica),
// transformed together as interleaved sequences so that a CTA holds ~512 points instead of
// a single warp's worth.
__global__ void __launch_bounds__(1024) batch_noise_rows_kernel(float2* data, const RepRec* __restrict__ recs,
                                                                int nx, int ny, int rows,
                                                                const float2* __restrict__ twx, float scale) {
    const long long row0 = (long long)blockIdx.x * rows;
    if (__ldg(&recs[row0 / ny].mode) != 2) return;
    extern __shared__ float2 sm[];
    float2* base = data + row0 * nx;
    const int log2n = 31 - __clz(nx);
    if (nx >= 256) {
        stockham_fft_io(sm, nx, log2n, 1, -1, twx, [&](int e) { return base[e]; },
                        [&](int e, float2 v) { base[e] = make_float2(v.x * scale, v.y * scale); });
        return;
    }
    // element j of row r at sm[fpad(j rows + r)]; global loads and stores stay row-contiguous
    const int lr = 31 - __clz(rows), total = rows * nx;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int r = i >> log2n, j = i & (nx - 1);
        sm[fpad((j << lr) + r)] = base[i];
    }
    stockham_fft(sm, nx, log2n, rows, -1, twx);
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int r = i >> log2n, j = i & (nx - 1);
        const float2 v = sm[fpad((j << lr) + r)];
        base[i] = make_float2(v.x * scale, v.y * scale);
    }
}

// --- spectra of a class ----------------------------------------------------------------

// z1 = drho + i jx, z2 = jy of every replica of the class (state of the current buffer)
// (the buffer holding the state is chosen by the parity of the device step counter, so a
// captured sample stays correct in every replay of its graph)
__global__ void batch_fields_kernel(const float* __restrict__ buf0, const float* __restrict__ buf1,
                                    const long long* __restrict__ kstep, long long rstride, Grid g, float2* z1,
                                    float2* z2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int rep = blockIdx.z;
    if (x >= g.nx) return;
    const float* src = ((__ldg(kstep) & 1) ? buf1 : buf0) + (long long)rep * rstride;
    const long long P = g.plane;
    const long long c = g.at(x, y);
    const float f0 = src[c], f1 = src[P + c - 1], f2 = src[2 * P + c - g.pitch], f3 = src[3 * P + c + 1];
    const float f4 = src[4 * P + c + g.pitch], f5 = src[5 * P + c - g.pitch - 1];
    const float f6 = src[6 * P + c - g.pitch + 1], f7 = src[7 * P + c + g.pitch + 1];
    const float f8 = src[8 * P + c + g.pitch - 1];
    const float drho = f0 + ((f1 + f3) + (f2 + f4)) + ((f5 + f7) + (f6 + f8));
    const float jx = (f1 - f3) + (f5 - f7) + (f8 - f6);
    const float jy = (f2 - f4) + (f5 - f7) + (f6 - f8);
    const long long o = ((long long)rep * g.ny + y) * g.nx + x;
    z1[o] = make_float2(drho, jx);
    z2[o] = make_float2(jy, 0.f);
}

__device__ __forceinline__ int ilog2b(int n) { return 31 - __clz(n); }

// forward row transforms of R*ny consecutive rows, scaled on the way out
__global__ void __launch_bounds__(1024) batch_rows_kernel(float2* data, int nx, const float2* __restrict__ twx,
                                                          float scale) {
    extern __shared__ float2 sm[];
    float2* rowp = data + (long long)blockIdx.x * nx;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) sm[fpad(j)] = rowp[j];
    stockham_fft(sm, nx, ilog2b(nx), 1, +1, twx);
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        const float2 v = sm[fpad(j)];
        rowp[j] = make_float2(v.x * scale, v.y * scale);
    }
}

// forward column transforms, strips of `count` columns, replica blockIdx.y
__global__ void __launch_bounds__(1024) batch_cols_kernel(float2* data, int nx, int ny, int count,
                                                          const float2* __restrict__ twy, float scale) {
    extern __shared__ float2 sm[];
    float2* base = data + (long long)blockIdx.y * nx * ny;
    const int xs = blockIdx.x * count;
    const int lc = 31 - __clz(count);
    const int total = ny * count;
    for (int e = threadIdx.x; e < total; e += blockDim.x)
        sm[fpad(e)] = base[(long long)(e >> lc) * nx + xs + (e & (count - 1))];
    stockham_fft(sm, ny, ilog2b(ny), count, +1, twy);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const float2 v = sm[fpad(e)];
        base[(long long)(e >> lc) * nx + xs + (e & (count - 1))] = make_float2(v.x * scale, v.y * scale);
    }
}

// per-replica radial bins (bins[rep][3][nbins]) from the class's bin table (lb_spectra.cuh;
// blockIdx.y = replica)
__global__ void batch_bin_kernel(const float2* __restrict__ z1, const float2* __restrict__ z2,
                                 const unsigned short* __restrict__ bin16, int nx, int ny, int nbins, double* bins) {
    extern __shared__ double sb[];
    for (int j = threadIdx.x; j < 3 * nbins; j += blockDim.x) sb[j] = 0.0;
    __syncthreads();
    const int rep = blockIdx.y;
    const long long n = (long long)nx * ny;
    const int wpb = blockDim.x >> 5;
    bin_half_plane(z1 + rep * n, z2 + rep * n, bin16, nx, ny, nbins, sb, blockIdx.x * wpb + (threadIdx.x >> 5),
                   gridDim.x * wpb);
    __syncthreads();
    double* out = bins + (long long)rep * 3 * nbins;
    for (int j = threadIdx.x; j < 3 * nbins; j += blockDim.x)
        if (sb[j] != 0.0) atomicAdd(&out[j], sb[j]);
}

// --- host side -------------------------------------------------------------------------

// Tile shapes the autotuner chooses from: (TX, TY, NT); TX * TY / NT nodes per thread.
static const int kBatchTiles[][3] = {{32, 16, 256}, {32, 16, 128}, {32, 8, 256}, {32, 8, 128},
                                     {64, 8, 256},  {64, 16, 512}, {32, 32, 512}};
constexpr int kBatchTileCount = 7;

static bool make_class_map(void* buf, const Grid& g, int R, int tile, CUtensorMap* map) {
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn || tile < 0 || tile >= kBatchTileCount) return false;
    cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * GY), (cuuint64_t)Q, (cuuint64_t)R};
    cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4, (cuuint64_t)g.plane * 4 * Q};
    // box: the tile plus 4 columns (16 bytes) on either side and one row above and below
    cuuint32_t box[4] = {(cuuint32_t)(kBatchTiles[tile][0] + 8), (cuuint32_t)(kBatchTiles[tile][1] + 2), 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    // 64-byte L2 promotion: a class's rows carry 128 bytes of ghost columns on either side of
    // which one 32-byte sector is ever written or read; with 256-byte promotion a box row
    // pulled whole rows of the small lattices (the 512-replica mix read 1.74x the algorithmic
    // bytes, 1.33x with 64; its 32^2 class 3.20x and 2.13x, 138 -> 112 us a step)
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// CTAs of a persistent launch: every SM filled to the occupancy the kernel allows
template <int TX, int TY, int NT, bool RS>
static cudaError_t ensemble_grid(int* grid) {
    using TT = TmaTile<TX, TY, float>;
    static GridCache cache;
    return resident_grid(step_ensemble_kernel<TX, TY, NT, RS>, NT, TT::SMEM_BYTES, cache, grid);
}

template <int TX, int TY, int NT>
static cudaError_t launch_ensemble_t(const EnsParams& p, cudaStream_t s) {
    using TT = TmaTile<TX, TY, float>;
    int grid = 0;
    cudaError_t e = p.rs ? ensemble_grid<TX, TY, NT, true>(&grid) : ensemble_grid<TX, TY, NT, false>(&grid);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(p.ntiles, grid));
    if (p.rs) step_ensemble_kernel<TX, TY, NT, true><<<blocks, NT, TT::SMEM_BYTES, s>>>(p);
    else step_ensemble_kernel<TX, TY, NT, false><<<blocks, NT, TT::SMEM_BYTES, s>>>(p);
    return cudaGetLastError();
}

static cudaError_t launch_ensemble(int tile, const EnsParams& p, cudaStream_t s) {
    switch (tile) {
        case 1: return launch_ensemble_t<32, 16, 128>(p, s);
        case 2: return launch_ensemble_t<32, 8, 256>(p, s);
        case 3: return launch_ensemble_t<32, 8, 128>(p, s);
        case 4: return launch_ensemble_t<64, 8, 256>(p, s);
        case 5: return launch_ensemble_t<64, 16, 512>(p, s);
        case 6: return launch_ensemble_t<32, 32, 512>(p, s);
        default: return launch_ensemble_t<32, 16, 256>(p, s);
    }
}

// prepares every kernel of the engine (attributes, occupancy) outside any stream capture
static cudaError_t prepare_ensemble_kernels() {
    int g = 0;
    cudaError_t e;
    for (int rs = 0; rs < 2; ++rs) {
        const bool R = rs != 0;
        if ((e = R ? ensemble_grid<32, 16, 256, true>(&g) : ensemble_grid<32, 16, 256, false>(&g)) != cudaSuccess) return e;
        if ((e = R ? ensemble_grid<32, 16, 128, true>(&g) : ensemble_grid<32, 16, 128, false>(&g)) != cudaSuccess) return e;
        if ((e = R ? ensemble_grid<32, 8, 256, true>(&g) : ensemble_grid<32, 8, 256, false>(&g)) != cudaSuccess) return e;
        if ((e = R ? ensemble_grid<32, 8, 128, true>(&g) : ensemble_grid<32, 8, 128, false>(&g)) != cudaSuccess) return e;
        if ((e = R ? ensemble_grid<64, 8, 256, true>(&g) : ensemble_grid<64, 8, 256, false>(&g)) != cudaSuccess) return e;
        if ((e = R ? ensemble_grid<64, 16, 512, true>(&g) : ensemble_grid<64, 16, 512, false>(&g)) != cudaSuccess) return e;
        if ((e = R ? ensemble_grid<32, 32, 512, true>(&g) : ensemble_grid<32, 32, 512, false>(&g)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Relaxation rates, Cholesky factors of Xi(0) (Sec. IV; the (4,9) block coupled unless
// noise_mode is LB_NOISE_DIAG) and noise switch of one lattice's record; the key, time
// offset and rho0/cs2 fields are left to the caller.
void fill_rep_record(double rho0, double cs2, double kT, double kappa, double tau_s, double tau_b,
                     double tau_ghost, int noise_mode, RepRec* rec) {
    double xi[81];
    lb_noise_matrix(rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost, 0.0, 0.0, xi);
    const double x44 = xi[3 * 9 + 3], x49 = noise_mode == LB_NOISE_DIAG ? 0.0 : xi[3 * 9 + 8], x99 = xi[8 * 9 + 8];
    const double L44 = std::sqrt(std::fmax(x44, 0.0));
    const double L94 = L44 > 0.0 ? x49 / L44 : 0.0;
    const double L99 = std::sqrt(std::fmax(x99 - L94 * L94, 0.0));
    rec->kappa = (float)kappa;
    rec->lb = (float)(-1.0 / tau_b);
    rec->ls = (float)(-1.0 / tau_s);
    rec->lq = rec->le = (float)(-1.0 / tau_ghost);
    rec->L44 = (float)L44; rec->L49 = 0.0f; rec->L94 = (float)L94; rec->L99 = (float)L99;
    rec->s5 = (float)std::sqrt(std::fmax(xi[4 * 9 + 4], 0.0));
    rec->s6 = (float)std::sqrt(std::fmax(xi[5 * 9 + 5], 0.0));
    rec->s7 = (float)std::sqrt(std::fmax(xi[6 * 9 + 6], 0.0));
    double co[6];
    noise_coefficients(rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost, co);
    rec->a44 = (float)co[0]; rec->b44 = (float)co[1];
    rec->a49 = (float)co[2]; rec->b49 = (float)co[3];
    rec->a99 = (float)co[4]; rec->b99 = (float)co[5];
    // real-space correlated noise: Cholesky factors of the (4,9) block at k^2 = 0, 4, 16/3, / 4
    const double sk[3] = {0.0, 4.0, 16.0 / 3.0};
    for (int j = 0; j < 3; ++j) {
        const double y44 = co[0] + co[1] * sk[j], y49 = co[2] + co[3] * sk[j], y99 = co[4] + co[5] * sk[j];
        const double l11 = std::sqrt(std::fmax(y44, 0.0));
        const double l21 = l11 > 0.0 ? y49 / l11 : 0.0;
        const double l22 = std::sqrt(std::fmax(y99 - l21 * l21, 0.0));
        rec->sL[j][0] = (float)(0.25 * l11); rec->sL[j][1] = 0.0f;
        rec->sL[j][2] = (float)(0.25 * l21); rec->sL[j][3] = (float)(0.25 * l22);
    }
    rec->mode = (noise_mode == LB_NOISE_OFF || kT <= 0.0)
                    ? 0
                    : (noise_mode == LB_NOISE_FULL ? 2 : (noise_mode == LB_NOISE_FULL_RS ? 3 : 1));
}

}  // namespace lbf

using namespace lbf;

namespace {

constexpr int kMaxBatchBins = 1024;
constexpr double SIGMA_S2_B = 1.0 / 3.0;

size_t align256b(size_t v) { return (v + 255) & ~size_t(255); }

bool pow2b(int v) { return v >= 2 && (v & (v - 1)) == 0; }

bool grid_of(int nx, int ny, Grid* g) {
    if (nx < 2 || ny < 2 || nx > 8192 || ny > 8192) return false;
    g->nx = nx; g->ny = ny; g->gx = 32;
    g->pitch = (nx + 64 + 31) / 32 * 32;
    g->plane = ((long long)g->pitch * (ny + 2 * GY) + 63) / 64 * 64;
    return true;
}

struct ClassInfo {
    int nx, ny, R;
    Grid g;
    std::vector<int> members;          // replica ids, in class order
    size_t off_buf[2], off_z1, off_z2, off_tw_x, off_tw_y, off_bin16, off_bins, off_counts, off_recs;
    size_t off_cosx, off_cosy;         // cos(2 pi m / n) tables of the correlated noise
    bool any_full = false;             // some replica of the class has correlated noise (k-space)
    bool any_rs = false;               // some replica of the class has correlated noise (real space)
};

struct Layout {
    std::vector<ClassInfo> classes;
    std::vector<int> cls_of, slot_of;  // replica -> class, index within the class
    size_t off_k, off_done, off_err, off_partial, off_sums, off_stage, off_fbar, total;
};

bool plan(int count, const int* nx, const int* ny, Layout* L) {
    std::map<std::pair<int, int>, int> index;
    L->classes.clear();
    L->cls_of.assign(count, 0);
    L->slot_of.assign(count, 0);
    size_t biggest = 0;
    for (int r = 0; r < count; ++r) {
        Grid g;
        if (!grid_of(nx[r], ny[r], &g)) return false;
        auto key = std::make_pair(nx[r], ny[r]);
        auto it = index.find(key);
        int c;
        if (it == index.end()) {
            c = (int)L->classes.size();
            index[key] = c;
            ClassInfo ci;
            ci.nx = nx[r]; ci.ny = ny[r]; ci.R = 0; ci.g = g;
            L->classes.push_back(ci);
        } else {
            c = it->second;
        }
        L->cls_of[r] = c;
        L->slot_of[r] = L->classes[c].R++;
        L->classes[c].members.push_back(r);
        biggest = std::max(biggest, (size_t)nx[r] * ny[r]);
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256b(off + bytes); return o; };
    for (auto& ci : L->classes) {
        const size_t n = (size_t)ci.nx * ci.ny;
        const size_t rbytes = (size_t)Q * ci.g.plane * sizeof(float) * ci.R;
        ci.off_buf[0] = take(rbytes);
        ci.off_buf[1] = take(rbytes);
        ci.off_z1 = take(n * ci.R * sizeof(float2));
        ci.off_z2 = take(n * ci.R * sizeof(float2));
        ci.off_tw_x = take(ci.nx * sizeof(float2));
        ci.off_tw_y = take(ci.ny * sizeof(float2));
        ci.off_bin16 = take(n * sizeof(unsigned short));
        ci.off_bins = take((size_t)ci.R * 3 * kMaxBatchBins * sizeof(double));
        ci.off_counts = take((size_t)kMaxBatchBins * sizeof(unsigned long long));
        ci.off_recs = take((size_t)ci.R * sizeof(RepRec));
        ci.off_cosx = take(ci.nx * sizeof(float));
        ci.off_cosy = take(ci.ny * sizeof(float));
    }
    L->off_k = take(sizeof(long long));
    L->off_done = take(sizeof(unsigned int));
    L->off_err = take(sizeof(int));
    L->off_partial = take((size_t)sums_partial_count() * sizeof(double));
    L->off_sums = take(3 * sizeof(double));
    L->off_stage = take(biggest * sizeof(double));
    L->off_fbar = take(Q * sizeof(double));
    L->total = off;
    return true;
}

}  // namespace

struct lb_batch {
    int count = 0, device = 0;
    double rho0 = 1.0, cs2 = SIGMA_S2_B;
    Layout L;
    char* ws = nullptr;
    bool owns = false;
    std::vector<RepRec> recs;              // host mirror, replica order
    std::vector<uint64_t> seeds;
    std::vector<long long> toff;
    std::vector<int> mode;                 // noise mode per replica (LB_NOISE_*)
    std::vector<bool> have_params;
    double fbar[Q];
    long long K = 0;                       // host mirror of the device step counter
    int every = 0, nbins = 0;
    long long nsamples = 0;
    std::vector<std::vector<unsigned long long>> counts;   // per class
    cudaStream_t stream = nullptr;
    std::string err;
    // captured graph of `graph_steps` steps
    cudaGraphExec_t graph = nullptr;
    long long graph_steps = 0;
    long long graph_kernels = 0;           // kernels one replay launches
    cudaStream_t cap_stream = nullptr;
    long long kernels = 0;
    // the step launches: up to MAX_CLASSES classes each, for tile shape `tile`
    int tile = 0;
    std::vector<EnsParams> launches;
    double autotune_ms = 0.0;              // per-step time of the chosen shape
};

static int bfail(lb_batch* b, int code, const std::string& m) {
    if (b) b->err = m; else set_context_free_error(m);
    return code;
}

#define BCK(b, call, where)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return bfail(b, LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static char* cls_ptr(lb_batch* b, size_t off) { return b->ws + off; }

static int upload_rec(lb_batch* b, int r) {
    const ClassInfo& ci = b->L.classes[b->L.cls_of[r]];
    RepRec* d = reinterpret_cast<RepRec*>(cls_ptr(b, ci.off_recs)) + b->L.slot_of[r];
    BCK(b, cudaMemcpyAsync(d, &b->recs[r], sizeof(RepRec), cudaMemcpyHostToDevice, b->stream), "H2D");
    return LB_OK;
}

// the multiplier and shift of div_magic for a divisor d >= 1
static void div_magic_params(int d, unsigned long long* m, int* s) {
    int l = 0;
    while ((1ll << l) < (long long)d) ++l;
    *s = 32 + l;
    *m = ((1ull << (32 + l)) + (unsigned long long)d - 1ull) / (unsigned long long)d;
}

// Kernel parameters of the step launches for tile shape `tile`: classes in chunks of
// MAX_CLASSES, the last launch of a step advancing the step counter.
static int build_launches(lb_batch* b, int tile, std::vector<EnsParams>* out) {
    out->clear();
    const int TX = kBatchTiles[tile][0], TY = kBatchTiles[tile][1];
    const int nc = (int)b->L.classes.size();
    for (int c0 = 0; c0 < nc; c0 += MAX_CLASSES) {
        EnsParams p;
        std::memset(&p, 0, sizeof(p));
        int tiles = 0;
        for (int j = 0; j < MAX_CLASSES && c0 + j < nc; ++j) {
            const ClassInfo& ci = b->L.classes[c0 + j];
            for (int w = 0; w < 2; ++w)
                if (!make_class_map(cls_ptr(b, ci.off_buf[w]), ci.g, ci.R, tile, &p.map[j][w]))
                    return bfail(b, LB_ECUDA, "cuTensorMapEncodeTiled failed for a size class");
            ClassDesc& d = p.cls[j];
            d.g = ci.g;
            d.buf[0] = reinterpret_cast<float*>(cls_ptr(b, ci.off_buf[0]));
            d.buf[1] = reinterpret_cast<float*>(cls_ptr(b, ci.off_buf[1]));
            d.recs = reinterpret_cast<const RepRec*>(cls_ptr(b, ci.off_recs));
            d.ntx = (ci.nx + TX - 1) / TX;
            d.per = d.ntx * ((ci.ny + TY - 1) / TY);
            div_magic_params(d.per, &d.per_m, &d.per_s);
            div_magic_params(d.ntx, &d.ntx_m, &d.ntx_s);
            d.tile_begin = tiles;
            d.rstride = (long long)Q * ci.g.plane;
            d.xi = reinterpret_cast<const float2*>(cls_ptr(b, ci.off_z1));
            const long long more = (long long)d.per * ci.R;
            if (tiles + more > (1ll << 30)) return bfail(b, LB_EINVAL, "too many tiles in one launch");
            tiles += (int)more;
            p.nclass = j + 1;
            p.rs = p.rs || ci.any_rs;
        }
        p.ntiles = tiles;
        p.kstep = reinterpret_cast<long long*>(cls_ptr(b, b->L.off_k));
        p.done = reinterpret_cast<unsigned int*>(cls_ptr(b, b->L.off_done));
        p.err = reinterpret_cast<int*>(cls_ptr(b, b->L.off_err));
        p.advance = 0;
        out->push_back(p);
    }
    if (!out->empty()) out->back().advance = 1;
    return LB_OK;
}

static int col_strip_b(int nx, int ny) {
    int c = 16;
    while (c > 1 && (fft_threads(ny, c) > 1024 || fft_smem_bytes(ny, c) > 200 * 1024)) c >>= 1;
    return c > nx ? nx : c;
}

// rows per CTA of the noise row pass: ~512 points for rows shorter than 256 (ny and the
// result powers of two, the result <= ny)
static int noise_rows_per_cta(int nx, int ny) {
    if (nx >= 256) return 1;
    int r = 512 / nx;
    return r > ny ? ny : r;
}

// correlated noise (xi_4, xi_9) of every correlated replica of class ci for the coming step,
// into the class's first spectra buffer (free between samples)
static int batch_noise(lb_batch* b, const ClassInfo& ci) {
    float2* xi = reinterpret_cast<float2*>(cls_ptr(b, ci.off_z1));
    const RepRec* recs = reinterpret_cast<const RepRec*>(cls_ptr(b, ci.off_recs));
    const int c = col_strip_b(ci.nx, ci.ny);
    batch_noise_cols_kernel<<<dim3(ci.nx / c, ci.R), fft_threads(ci.ny, c), fft_smem_bytes(ci.ny, c), b->stream>>>(
        xi, recs, reinterpret_cast<const long long*>(cls_ptr(b, b->L.off_k)), ci.nx, ci.ny, c,
        reinterpret_cast<const float2*>(cls_ptr(b, ci.off_tw_y)), reinterpret_cast<const float*>(cls_ptr(b, ci.off_cosx)),
        reinterpret_cast<const float*>(cls_ptr(b, ci.off_cosy)));
    const float scale = (float)(1.0 / std::sqrt((double)ci.nx * ci.ny));
    const int rows = noise_rows_per_cta(ci.nx, ci.ny);
    batch_noise_rows_kernel<<<ci.R * ci.ny / rows, fft_threads(ci.nx, rows), fft_smem_bytes(ci.nx, rows),
                              b->stream>>>(xi, recs, ci.nx, ci.ny, rows,
                                           reinterpret_cast<const float2*>(cls_ptr(b, ci.off_tw_x)), scale);
    BCK(b, cudaGetLastError(), "correlated noise");
    b->kernels += 2;
    return LB_OK;
}

static int batch_step_eager(lb_batch* b) {
    for (const ClassInfo& ci : b->L.classes)
        if (ci.any_full) {
            int r = batch_noise(b, ci);
            if (r != LB_OK) return r;
        }
    for (const EnsParams& p : b->launches) {
        BCK(b, launch_ensemble(b->tile, p, b->stream), "ensemble step");
        b->kernels++;
    }
    return LB_OK;
}

static int batch_sample(lb_batch* b, cudaStream_t s) {
    for (auto& ci : b->L.classes) {
        float2* z1 = reinterpret_cast<float2*>(cls_ptr(b, ci.off_z1));
        float2* z2 = reinterpret_cast<float2*>(cls_ptr(b, ci.off_z2));
        dim3 grd((ci.nx + 127) / 128, ci.ny, ci.R);
        batch_fields_kernel<<<grd, 128, 0, s>>>(reinterpret_cast<const float*>(cls_ptr(b, ci.off_buf[0])),
                                                reinterpret_cast<const float*>(cls_ptr(b, ci.off_buf[1])),
                                                reinterpret_cast<const long long*>(cls_ptr(b, b->L.off_k)),
                                                (long long)Q * ci.g.plane, ci.g, z1, z2);
        const float scale = (float)(1.0 / std::sqrt((double)ci.nx * ci.ny));
        const float2* twx = reinterpret_cast<const float2*>(cls_ptr(b, ci.off_tw_x));
        const float2* twy = reinterpret_cast<const float2*>(cls_ptr(b, ci.off_tw_y));
        const size_t rsm = fft_smem_bytes(ci.nx, 1);
        const int c = col_strip_b(ci.nx, ci.ny);
        const size_t csm = fft_smem_bytes(ci.ny, c);
        for (float2* z : {z1, z2}) {
            batch_rows_kernel<<<ci.R * ci.ny, fft_threads(ci.nx, 1), rsm, s>>>(z, ci.nx, twx, 1.0f);
            batch_cols_kernel<<<dim3(ci.nx / c, ci.R), fft_threads(ci.ny, c), csm, s>>>(z, ci.nx, ci.ny, c, twy, scale);
        }
        const size_t bsm = (size_t)3 * b->nbins * sizeof(double);
        const int units = (ci.ny / 2 + 1) * ((ci.nx / 2 + 32) / 32);   // warp work units per replica
        const int bx = std::max(1, std::min(64, units / 32));
        batch_bin_kernel<<<dim3(bx, ci.R), 256, bsm, s>>>(z1, z2, reinterpret_cast<const unsigned short*>(cls_ptr(b, ci.off_bin16)),
                                                          ci.nx, ci.ny, b->nbins, reinterpret_cast<double*>(cls_ptr(b, ci.off_bins)));
        BCK(b, cudaGetLastError(), "spectra sample");
        b->kernels += 6;
    }
    return LB_OK;
}

// one step (kernels, counter advance, optional sample) issued on stream s
static int batch_one_step(lb_batch* b, cudaStream_t s) {
    cudaStream_t keep = b->stream;
    b->stream = s;
    int r = batch_step_eager(b);
    if (r == LB_OK) {
        b->K++;
        if (b->every > 0 && b->K % b->every == 0) {
            r = batch_sample(b, s);
            b->nsamples++;
        }
    }
    b->stream = keep;
    return r;
}

extern "C" {

size_t lb_batch_workspace_bytes(int count, const int* nx, const int* ny) {
    if (count < 1 || !nx || !ny) return 0;
    Layout L;
    if (!plan(count, nx, ny, &L)) return 0;
    return L.total;
}

int lb_batch_create(int count, const int* nx, const int* ny, const uint64_t* seeds, double rho0, double cs2,
                    void* workspace, size_t workspace_bytes, lb_batch** out) {
    if (!out || count < 1 || !nx || !ny || !seeds) return bfail(nullptr, LB_EINVAL, "invalid arguments");
    *out = nullptr;
    if (!(rho0 > 0.0) || !(cs2 > 0.0)) return bfail(nullptr, LB_EINVAL, "rho0 and cs2 must be positive");
    lb_batch* b = new lb_batch();
    if (!plan(count, nx, ny, &b->L)) {
        delete b;
        return bfail(nullptr, LB_EINVAL, "every lattice side must lie in [2, 8192]");
    }
    b->count = count;
    b->rho0 = rho0;
    b->cs2 = cs2;
    cudaGetDevice(&b->device);
    if (workspace) {
        if (workspace_bytes < b->L.total || ((uintptr_t)workspace & 255)) {
            delete b;
            return bfail(nullptr, LB_ENOMEM, "workspace smaller than lb_batch_workspace_bytes() or misaligned");
        }
        b->ws = (char*)workspace;
    } else {
        cudaError_t e = cudaMalloc((void**)&b->ws, b->L.total);
        if (e != cudaSuccess) {
            delete b;
            return bfail(nullptr, LB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        b->owns = true;
    }
    rest_populations(rho0, cs2, b->fbar);
    b->seeds.assign(seeds, seeds + count);
    b->recs.assign(count, RepRec{});
    b->toff.assign(count, 0);
    b->mode.assign(count, LB_NOISE_OFF);
    b->have_params.assign(count, false);
    for (int r = 0; r < count; ++r) {
        RepRec& rc = b->recs[r];
        rc.rho0 = (float)rho0;
        rc.cs2m = (float)(cs2 - SIGMA_S2_B);
        rc.lb = rc.ls = rc.lq = rc.le = -1.0f;
        rc.k0 = (uint32_t)(seeds[r] & 0xffffffffu);
        rc.k1 = (uint32_t)(seeds[r] >> 32);
    }
    cudaError_t e = cudaMemset(b->ws, 0, b->L.total);
    std::vector<float2> tw;
    size_t noise_csm = 0, noise_rsm = 0;
    for (auto& ci : b->L.classes) {
        if (e != cudaSuccess) break;
        for (int which = 0; which < 2; ++which) {
            const int n = which == 0 ? ci.nx : ci.ny;
            tw.resize(n);
            for (int k = 0; k < n; ++k) {
                const double a = 2.0 * M_PI * (double)k / n;
                tw[k] = make_float2((float)std::cos(a), (float)-std::sin(a));
            }
            e = cudaMemcpy(cls_ptr(b, which == 0 ? ci.off_tw_x : ci.off_tw_y), tw.data(), n * sizeof(float2),
                           cudaMemcpyHostToDevice);
            if (e != cudaSuccess) break;
            std::vector<float> cs(n);
            for (int k = 0; k < n; ++k) cs[k] = (float)std::cos(2.0 * M_PI * (double)k / n);
            e = cudaMemcpy(cls_ptr(b, which == 0 ? ci.off_cosx : ci.off_cosy), cs.data(), n * sizeof(float),
                           cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && pow2b(ci.nx) && pow2b(ci.ny) && ci.ny <= 8192) {
            // shared memory of the correlated-noise kernels, set before any graph capture
            const int c = col_strip_b(ci.nx, ci.ny);
            noise_csm = std::max(noise_csm, fft_smem_bytes(ci.ny, c));
            noise_rsm = std::max(noise_rsm, fft_smem_bytes(ci.nx, noise_rows_per_cta(ci.nx, ci.ny)));
        }
    }
    for (int r = 0; r < count && e == cudaSuccess; ++r) {
        const ClassInfo& ci = b->L.classes[b->L.cls_of[r]];
        e = cudaMemcpy(reinterpret_cast<RepRec*>(cls_ptr(b, ci.off_recs)) + b->L.slot_of[r], &b->recs[r],
                       sizeof(RepRec), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(cls_ptr(b, b->L.off_fbar), b->fbar, sizeof(double) * Q, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = prepare_ensemble_kernels();
    if (e == cudaSuccess && noise_csm > 0)
        e = cudaFuncSetAttribute(batch_noise_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)noise_csm);
    if (e == cudaSuccess && noise_rsm > 0)
        e = cudaFuncSetAttribute(batch_noise_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)noise_rsm);
    {
        // LBFLUCT_BATCH_TILE=<0..6> fixes the tile shape until an autotune (tests of every shape)
        const char* tv = std::getenv("LBFLUCT_BATCH_TILE");
        const int t = tv ? std::atoi(tv) : 0;
        b->tile = (t >= 0 && t < kBatchTileCount) ? t : 0;
    }
    if (e == cudaSuccess && build_launches(b, b->tile, &b->launches) != LB_OK) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        if (b->owns) cudaFree(b->ws);
        delete b;
        return bfail(nullptr, LB_ECUDA, std::string("lb_batch_create: ") + cudaGetErrorString(e));
    }
    *out = b;
    return LB_OK;
}

int lb_batch_destroy(lb_batch* b) {
    if (!b) return LB_EINVAL;
    DeviceGuard dg(b->device);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->owns) cudaFree(b->ws);
    delete b;
    return LB_OK;
}

int lb_batch_set_stream(lb_batch* b, void* stream) {
    if (!b) return LB_EINVAL;
    b->stream = (cudaStream_t)stream;
    return LB_OK;
}

int lb_batch_set_params(lb_batch* b, int replica, double kT, double kappa, double tau_s, double tau_b,
                        double tau_ghost, int noise_mode) {
    if (!b || replica < -1 || replica >= b->count) return LB_EINVAL;
    DeviceGuard dg(b->device);
    const int lo = replica < 0 ? 0 : replica, hi = replica < 0 ? b->count : replica + 1;
    if (noise_mode == LB_NOISE_LW_LOCAL)
        return bfail(b, LB_EINVAL, "the batched engine steps homogeneous noise modes only (not LB_NOISE_LW_LOCAL)");
    for (int r = lo; r < hi; ++r) {
        const ClassInfo& ci = b->L.classes[b->L.cls_of[r]];
        if (noise_mode == LB_NOISE_FULL &&
            (!pow2b(ci.nx) || !pow2b(ci.ny) || ci.ny > 8192 || col_strip_b(ci.nx, ci.ny) < 2))
            return bfail(b, LB_EINVAL, "correlated noise needs nx and ny powers of two and ny <= 8192");
        int rc = lb_check_params(ci.nx, ci.ny, b->rho0, b->cs2, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode);
        if (rc != LB_OK) return bfail(b, rc, "parameters rejected (see lb_check_params)");
    }
    for (int r = lo; r < hi; ++r) {
        fill_rep_record(b->rho0, b->cs2, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode, &b->recs[r]);
        b->mode[r] = noise_mode;
        b->have_params[r] = true;
        int u = upload_rec(b, r);
        if (u != LB_OK) return u;
    }
    // classes that now need (or no longer need) the correlated-noise kernels, or the step
    // kernel variant with real-space correlated noise
    bool changed = false, changed_rs = false;
    for (auto& ci : b->L.classes) {
        bool any = false, any_rs = false;
        for (int r : ci.members) {
            any = any || b->recs[r].mode == 2;
            any_rs = any_rs || b->recs[r].mode == 3;
        }
        changed = changed || any != ci.any_full;
        changed_rs = changed_rs || any_rs != ci.any_rs;
        ci.any_full = any;
        ci.any_rs = any_rs;
    }
    if (changed_rs) {
        int rc = build_launches(b, b->tile, &b->launches);
        if (rc != LB_OK) return rc;
        changed = true;
    }
    if (changed && b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; b->graph_steps = 0; }
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_batch_autotune(lb_batch* b, int steps) {
    if (!b || steps < 1) return LB_EINVAL;
    DeviceGuard dg(b->device);
    for (int r = 0; r < b->count; ++r)
        if (!b->have_params[r]) return bfail(b, LB_ESTATE, "lb_batch_set_params must be called for every replica");
    // times each tile shape on the whole ensemble (launches that leave the step counter
    // alone), keeps the fastest, then puts every replica back at rest at K = 0
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
    } ev;
    BCK(b, cudaEventCreate(&ev.a), "event");
    BCK(b, cudaEventCreate(&ev.b), "event");
    float best = 1e30f;
    int best_tile = 0;
    std::vector<EnsParams> cand;
    for (int t = 0; t < kBatchTileCount; ++t) {
        int rc = build_launches(b, t, &cand);
        if (rc != LB_OK) return rc;
        for (auto& p : cand) p.advance = 0;
        for (const auto& p : cand) BCK(b, launch_ensemble(t, p, b->stream), "autotune");   // warm-up
        // the fastest of three timed runs of `steps` steps (a single short run is at the
        // mercy of clock ramps and of whatever else the device is finishing)
        for (int rep = 0; rep < 3; ++rep) {
            BCK(b, cudaEventRecord(ev.a, b->stream), "event");
            for (int k = 0; k < steps; ++k)
                for (const auto& p : cand) BCK(b, launch_ensemble(t, p, b->stream), "autotune");
            BCK(b, cudaEventRecord(ev.b, b->stream), "event");
            BCK(b, cudaEventSynchronize(ev.b), "event");
            float ms = 0.f;
            BCK(b, cudaEventElapsedTime(&ms, ev.a, ev.b), "event");
            if (ms < best) { best = ms; best_tile = t; }
        }
        b->kernels += (long long)(3 * steps + 1) * (long long)cand.size();
    }
    b->tile = best_tile;
    int rc = build_launches(b, best_tile, &b->launches);
    if (rc != LB_OK) return rc;
    b->autotune_ms = best / steps;
    for (auto& ci : b->L.classes) {
        BCK(b, cudaMemsetAsync(cls_ptr(b, ci.off_buf[0]), 0, (size_t)Q * ci.g.plane * 4 * ci.R, b->stream), "memset");
        BCK(b, cudaMemsetAsync(cls_ptr(b, ci.off_buf[1]), 0, (size_t)Q * ci.g.plane * 4 * ci.R, b->stream), "memset");
    }
    BCK(b, cudaMemsetAsync(cls_ptr(b, b->L.off_k), 0, sizeof(long long), b->stream), "memset");
    b->K = 0;
    for (int r = 0; r < b->count; ++r) {
        b->toff[r] = 0;
        b->recs[r].toff = 0;
        int u = upload_rec(b, r);
        if (u != LB_OK) return u;
    }
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; b->graph_steps = 0; }
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_batch_step(lb_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return LB_EINVAL;
    DeviceGuard dg(b->device);
    for (int r = 0; r < b->count; ++r)
        if (!b->have_params[r]) return bfail(b, LB_ESTATE, "lb_batch_set_params must be called for every replica");
    for (int64_t k = 0; k < nsteps; ++k) {
        int r = batch_one_step(b, b->stream);
        if (r != LB_OK) return r;
    }
    return LB_OK;
}

int lb_batch_step_graph(lb_batch* b, int64_t nsteps, int64_t steps_per_graph) {
    if (!b || nsteps < 0 || steps_per_graph < 1) return LB_EINVAL;
    DeviceGuard dg(b->device);
    for (int r = 0; r < b->count; ++r)
        if (!b->have_params[r]) return bfail(b, LB_ESTATE, "lb_batch_set_params must be called for every replica");
    const long long G = steps_per_graph;
    if (b->every > 0 && G % b->every != 0) return bfail(b, LB_EINVAL, "steps_per_graph must be a multiple of every");
    // eager steps until the graph's samples fall on multiples of `every`
    while (nsteps > 0 && b->every > 0 && b->K % b->every != 0) {
        int r = batch_one_step(b, b->stream);
        if (r != LB_OK) return r;
        --nsteps;
    }
    if (nsteps >= G && (!b->graph || b->graph_steps != G)) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        if (!b->cap_stream) BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream");
        const long long K0 = b->K, n0 = b->nsamples, k0 = b->kernels;
        BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
        int rc = LB_OK;
        for (long long k = 0; k < G && rc == LB_OK; ++k) rc = batch_one_step(b, b->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
        b->K = K0; b->nsamples = n0;               // capture issued nothing; the replays will
        const long long per_graph = b->kernels - k0;
        b->kernels = k0;
        if (rc != LB_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return bfail(b, LB_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(b, LB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->graph_steps = G;
        b->graph_kernels = per_graph;
    }
    while (nsteps >= G && b->graph) {
        BCK(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
        b->K += G;
        if (b->every > 0) b->nsamples += G / b->every;
        b->kernels += b->graph_kernels;
        nsteps -= G;
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        int r = batch_one_step(b, b->stream);
        if (r != LB_OK) return r;
    }
    return LB_OK;
}

int lb_batch_get_time(lb_batch* b, int replica, int64_t* t) {
    if (!b || !t || replica < 0 || replica >= b->count) return LB_EINVAL;
    *t = b->K + b->toff[replica];
    return LB_OK;
}

static void* rep_pops(lb_batch* b, int r, int which) {
    const ClassInfo& ci = b->L.classes[b->L.cls_of[r]];
    return cls_ptr(b, ci.off_buf[which]) + (size_t)b->L.slot_of[r] * Q * ci.g.plane * sizeof(float);
}

int lb_batch_set_populations(lb_batch* b, int replica, const double* f, int loc, int64_t t) {
    if (!b || !f || replica < 0 || replica >= b->count || (loc != LB_HOST && loc != LB_DEVICE) || t < 0)
        return LB_EINVAL;
    DeviceGuard dg(b->device);
    const ClassInfo& ci = b->L.classes[b->L.cls_of[replica]];
    const long long n = (long long)ci.nx * ci.ny;
    double* stage = reinterpret_cast<double*>(cls_ptr(b, b->L.off_stage));
    void* pops = rep_pops(b, replica, (int)(b->K & 1));
    for (int i = 0; i < Q; ++i) {
        const double* src = f + i * n;
        if (loc == LB_HOST) {
            BCK(b, cudaMemcpyAsync(stage, src, sizeof(double) * n, cudaMemcpyHostToDevice, b->stream), "H2D");
            src = stage;
        }
        BCK(b, launch_set_plane(src, pops, 0, ci.g, i, b->fbar[i], b->stream), "set populations");
        b->kernels++;
    }
    b->toff[replica] = t - b->K;
    b->recs[replica].toff = b->toff[replica];
    int u = upload_rec(b, replica);
    if (u != LB_OK) return u;
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_batch_get_populations(lb_batch* b, int replica, double* f, int loc) {
    if (!b || !f || replica < 0 || replica >= b->count || (loc != LB_HOST && loc != LB_DEVICE)) return LB_EINVAL;
    DeviceGuard dg(b->device);
    const ClassInfo& ci = b->L.classes[b->L.cls_of[replica]];
    const long long n = (long long)ci.nx * ci.ny;
    double* stage = reinterpret_cast<double*>(cls_ptr(b, b->L.off_stage));
    const void* pops = rep_pops(b, replica, (int)(b->K & 1));
    for (int i = 0; i < Q; ++i) {
        double* dst = loc == LB_HOST ? stage : f + i * n;
        BCK(b, launch_get_plane(pops, 0, ci.g, i, b->fbar[i], dst, b->stream), "get populations");
        b->kernels++;
        if (loc == LB_HOST)
            BCK(b, cudaMemcpyAsync(f + i * n, stage, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream), "D2H");
    }
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    int h = 0;
    BCK(b, cudaMemcpy(&h, cls_ptr(b, b->L.off_err), sizeof(int), cudaMemcpyDeviceToHost), "D2H");
    if (h) return bfail(b, LB_ETIMEOUT, "a batched step kernel gave up waiting for its TMA loads");
    return LB_OK;
}

int lb_batch_sums(lb_batch* b, int replica, double sums[3]) {
    if (!b || !sums || replica < 0 || replica >= b->count) return LB_EINVAL;
    DeviceGuard dg(b->device);
    const ClassInfo& ci = b->L.classes[b->L.cls_of[replica]];
    double* partial = reinterpret_cast<double*>(cls_ptr(b, b->L.off_partial));
    double* s3 = reinterpret_cast<double*>(cls_ptr(b, b->L.off_sums));
    BCK(b, launch_sums(rep_pops(b, replica, (int)(b->K & 1)), 0, ci.g,
                       reinterpret_cast<const double*>(cls_ptr(b, b->L.off_fbar)), partial, s3, b->stream), "sums");
    b->kernels += 2;
    BCK(b, cudaMemcpyAsync(sums, s3, 3 * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "D2H");
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_batch_set_sampling(lb_batch* b, int every, int nbins) {
    if (!b || every < 0) return LB_EINVAL;
    DeviceGuard dg(b->device);
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; b->graph_steps = 0; }
    if (every == 0) { b->every = 0; return LB_OK; }
    if (nbins < 1 || nbins > kMaxBatchBins) return bfail(b, LB_EINVAL, "nbins must lie in [1, 1024]");
    size_t rsm = 0, csm = 0;
    for (auto& ci : b->L.classes) {
        if (!pow2b(ci.nx) || !pow2b(ci.ny)) return bfail(b, LB_EINVAL, "spectra need power-of-two lattice sides");
        rsm = std::max(rsm, fft_smem_bytes(ci.nx, 1));
        csm = std::max(csm, fft_smem_bytes(ci.ny, col_strip_b(ci.nx, ci.ny)));
    }
    // shared memory of the sample kernels, set here so that a graph capture makes no such call
    BCK(b, cudaFuncSetAttribute(batch_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm), "attr");
    BCK(b, cudaFuncSetAttribute(batch_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm), "attr");
    BCK(b, cudaFuncSetAttribute(batch_bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(3 * nbins * sizeof(double))), "attr");
    b->every = every;
    b->nbins = nbins;
    b->nsamples = 0;
    b->counts.assign(b->L.classes.size(), std::vector<unsigned long long>(nbins, 0));
    for (size_t c = 0; c < b->L.classes.size(); ++c) {
        ClassInfo& ci = b->L.classes[c];
        BCK(b, cudaMemsetAsync(cls_ptr(b, ci.off_bins), 0, (size_t)ci.R * 3 * kMaxBatchBins * sizeof(double),
                               b->stream), "memset");
        BCK(b, launch_bin_counts(ci.nx, ci.ny, nbins, reinterpret_cast<unsigned short*>(cls_ptr(b, ci.off_bin16)),
                                 reinterpret_cast<unsigned long long*>(cls_ptr(b, ci.off_counts)), b->stream), "bins");
        BCK(b, cudaMemcpyAsync(b->counts[c].data(), cls_ptr(b, ci.off_counts), nbins * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, b->stream), "D2H");
    }
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_batch_structure_factor(lb_batch* b, int replica, int nbins, double* S_rho, double* S_jl, double* S_jt,
                              int64_t* counts, int64_t* nsamples) {
    if (!b || replica < 0 || replica >= b->count) return LB_EINVAL;
    DeviceGuard dg(b->device);
    if (nbins != b->nbins || b->nbins == 0) return bfail(b, LB_EINVAL, "nbins differs from lb_batch_set_sampling");
    const int c = b->L.cls_of[replica];
    const ClassInfo& ci = b->L.classes[c];
    std::vector<double> h(3 * (size_t)nbins);
    const double* src = reinterpret_cast<const double*>(cls_ptr(b, ci.off_bins)) + (size_t)b->L.slot_of[replica] * 3 * nbins;
    BCK(b, cudaMemcpyAsync(h.data(), src, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "D2H");
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    for (int k = 0; k < nbins; ++k) {
        const double den = (double)b->counts[c][k] * (double)b->nsamples;
        if (S_rho) S_rho[k] = den > 0 ? h[k] / den : 0.0;
        if (S_jl) S_jl[k] = den > 0 ? h[nbins + k] / den : 0.0;
        if (S_jt) S_jt[k] = den > 0 ? h[2 * nbins + k] / den : 0.0;
        if (counts) counts[k] = (int64_t)b->counts[c][k];
    }
    if (nsamples) *nsamples = b->nsamples;
    return LB_OK;
}

int lb_batch_launch_count(lb_batch* b, int64_t* n) {
    if (!b || !n) return LB_EINVAL;
    *n = b->kernels;
    return LB_OK;
}

int lb_batch_tuning(lb_batch* b, int* tile_x, int* tile_y, int* threads, double* ms_per_step) {
    if (!b) return LB_EINVAL;
    if (tile_x) *tile_x = kBatchTiles[b->tile][0];
    if (tile_y) *tile_y = kBatchTiles[b->tile][1];
    if (threads) *threads = kBatchTiles[b->tile][2];
    if (ms_per_step) *ms_per_step = b->autotune_ms;
    return LB_OK;
}

const char* lb_batch_last_error(lb_batch* b) { return b ? b->err.c_str() : lb_last_error(nullptr); }

}  // extern "C"
