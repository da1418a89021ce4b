// lb_step_tma.cu -- the fused fluctuating D2Q9 step, TMA-staged and persistent.
//
// Same arithmetic as lb_step.cu (collide_node), different data movement:
//   * a persistent grid (resident CTAs only) walks the lattice in TX x TY tiles (the shape
//     chosen per noise mode and storage, tma_default_tile) in row-major tile order, so the
//     tiles in flight form a band whose halo rows are still in L2 when the neighbouring tile
//     reads them;
//   * for each tile one thread issues nine 3D TMA loads (cp.async.bulk.tensor), one per
//     population plane, of the box [x0 - 4, x0 + TX + 4) x [y0 - 1 - cy_i, y0 + TY + 1 - cy_i)
//     into shared memory; the y offset of plane i absorbs its streaming shift, so node
//     (lx, ly) of the tile reads f_i at box[ly + 1][lx + 4 - cx_i].  The x start is rounded
//     down to a 16-byte boundary (four floats) as TMA requires;
//   * two stages and an mbarrier each: tile k+1 is in flight while tile k is computed;
//   * every thread pulls its nodes' nine deviations from shared memory into registers and
//     writes their density to a tile-plus-ring array (the ring from the halo); after one
//     barrier the stage is refilled with the tile two steps ahead while every node
//     collides and stores its nine post-collision deviations (and periodic ghosts)
//     directly from registers with coalesced stores.  Nodes beyond a ragged edge of the
//     lattice take part in the density pass (their values are never used) but not in the
//     collision pass.
// Waits on the mbarriers are bounded by the global timer; a CTA that gives up sets the
// error word, gives its loads in flight a bounded chance to land, and returns.
#include <cuda.h>

#include <type_traits>

#include "lb_collide.cuh"
#include "lb_tma.cuh"

namespace lbf {

struct TmaArgs {
    StepArgs a;
    int ntx, nty;      // tiles along x and y
    int* err;          // device error word (1 = a TMA wait timed out)
};


// POLY: the double-well equation of state (the bulk pressure's quartic in drho, StepArgs e2..e4)
template <int TX, int TY, int NT, int MODE, typename T, bool POLY = false>
__global__ void __launch_bounds__(NT) step_tma_kernel(const __grid_constant__ CUtensorMap tmap, const TmaArgs ta) {
    using TT = TmaTile<TX, TY, T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* smem = reinterpret_cast<T*>(smem_raw);
    float* R = reinterpret_cast<float*>(smem_raw + 2 * TT::STAGE_BYTES);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(R + TT::RW * TT::RH);
    const StepArgs& a = ta.a;
    const Grid g = a.g;
    const int tid = threadIdx.x;
    const int ntiles = ta.ntx * ta.nty;
    // FP16 storage collides in the stored form g_i = df_i / w_i (no scaling on load or store)
    constexpr bool GF = std::is_same<T, __half>::value;
    auto load9 = [](const T* S, int b, float f[Q]) { load9_ps<TT::PS, T, GF>(S, b, f); };
    auto rho_of = [](const float f[Q]) { return GF ? drho_of_g(f) : drho_of(f); };
    // MODE 3: the 2 x 2-box noise contributions, after the mbarriers (kept apart from the
    // stages: filling them into the consumed stage and refilling it after the collision
    // measured slower, the two extra barriers costing more than the fourth CTA per SM gained)
    float2* H = reinterpret_cast<float2*>(smem_raw + TT::H_OFFSET);

    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    }
    __syncthreads();

    // the nine boxes of the tile in column col, row row of the tiling into stage s
    auto issue = [&](int col, int row, int s) {
        const int x0 = col * TX, y0 = row * TY;
        const uint32_t bar = smem_u32(&mbar[s]);
        mbar_expect_tx(bar, TT::TX_BYTES);
        T* st = smem + s * TT::STAGE;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            tma_load_3d(smem_u32(st + i * TT::PS), &tmap, x0 - TT::XO + g.gx, y0 - 1 - kCYt[i] + GY, i, bar);
    };

    // a tile's column and row, advanced by the grid stride without a division per tile
    const int first = blockIdx.x;
    const int stx = (int)gridDim.x % ta.ntx, sty = (int)gridDim.x / ta.ntx;
    auto advance = [&](int& col, int& row) {
        col += stx;
        row += sty;
        if (col >= ta.ntx) {
            col -= ta.ntx;
            ++row;
        }
    };
    int tcol = first % ta.ntx, trow = first / ta.ntx;
    if (tid == 0) {
        if (first < ntiles) issue(tcol, trow, 0);
        int c1 = tcol, r1 = trow;
        advance(c1, r1);
        if (first + (int)gridDim.x < ntiles) issue(c1, r1, 1);
    }
    int k = 0;
    for (int tile = first; tile < ntiles; tile += gridDim.x, ++k) {
        const int s = k & 1;
        const uint32_t parity = (uint32_t)((k >> 1) & 1);
        // bounded wait for this tile's nine boxes; the decision to give up is collective
        // (this barrier also orders the previous tile's reads of R before this tile's writes)
        const bool ok = mbar_wait_bounded(smem_u32(&mbar[s]), parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(ta.err, 1);
                // give the loads still in flight into this CTA's shared memory a bounded
                // chance to land before the CTA exits
                mbar_wait_bounded(smem_u32(&mbar[s]), parity);
                if (tile + (int)gridDim.x < ntiles)
                    mbar_wait_bounded(smem_u32(&mbar[s ^ 1]), (uint32_t)(((k + 1) >> 1) & 1));
            }
            return;
        }
        const T* S = smem + s * TT::STAGE;
        const int x0 = tcol * TX, y0 = trow * TY;
        advance(tcol, trow);        // now the next tile's

        static_assert((TX * TY) % NT == 0, "tile must be a multiple of the block");
        constexpr int NN = TX * TY / NT;
        // each thread pulls its nodes' nine deviations once, keeps them in registers across
        // the barrier and writes their density to the tile; the ring is formed separately
        float fr[NN][Q];
#pragma unroll
        for (int it = 0; it < NN; ++it) {
            const int q = tid + it * NT;
            const int ly = q / TX, lx = q - ly * TX;
            load9(S, (ly + 1) * TT::BW + lx + TT::XO, fr[it]);
            R[(ly + 1) * TT::RW + lx + 1] = rho_of(fr[it]);
        }
        // real-space correlated noise: every node's contributions, then the halo's
        auto stencil_tile = [&](float2* Hd) {
#pragma unroll 1
            for (int it = 0; it < NN; ++it) {
                const int q = tid + it * NT;
                const int ly = q / TX, lx = q - ly * TX;
                const int x = x0 + lx, y = y0 + ly;
                if (x < g.nx && y < g.ny)
                    stencil_store<TT::HW>(a, Hd, TT::HN, lx, ly, (uint32_t)y * (uint32_t)g.nx + (uint32_t)x);
            }
            stencil_halo<TX, TY, TT::HW>(a, Hd, TT::HN, x0, y0, g.nx, g.ny, tid, NT);
        };
        if (MODE == 3) stencil_tile(H);
        // the ring: rows 0 and TY + 1 (TX + 2 each), then columns 0 and TX + 1, on the last
        // threads (the first issues the refill); with MODE 3 on the first (the last form the
        // noise contributions of the halo)
        constexpr int NB = 2 * (TX + 2) + 2 * TY;
        for (int j = MODE == 3 ? tid : NT - 1 - tid; j < NB; j += NT) {
            int rx, ry;
            if (j < TX + 2) { rx = j; ry = 0; }
            else if (j < 2 * (TX + 2)) { rx = j - (TX + 2); ry = TY + 1; }
            else { const int u = j - 2 * (TX + 2); ry = 1 + (u >> 1); rx = (u & 1) ? TX + 1 : 0; }
            float h[Q];
            load9(S, ry * TT::BW + rx + TT::XO - 1, h);
            R[ry * TT::RW + rx] = rho_of(h);
        }
        __syncthreads();
        // the collision pass reads no population from stage s: refill it now with the tile
        // two steps ahead
        if (tid == 0 && tile + 2 * (int)gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            int c2 = tcol, r2 = trow;
            advance(c2, r2);
            issue(c2, r2, s);
        }

        // collide every node of the tile; the nodes of one thread are independent, so
        // their random-number and collision chains interleave
#pragma unroll
        for (int it = 0; it < NN; ++it) {
            const int q = tid + it * NT;
            const int ly = q / TX, lx = q - ly * TX;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= g.nx || y >= g.ny) continue;
            const float* f = fr[it];
            const int rc = (ly + 1) * TT::RW + lx + 1;
            Nbr r;
            r.C = R[rc];
            r.E = R[rc + 1]; r.W = R[rc - 1];
            r.N = R[rc + TT::RW]; r.S = R[rc - TT::RW];
            r.NE = R[rc + TT::RW + 1]; r.NW = R[rc + TT::RW - 1];
            r.SE = R[rc - TT::RW + 1]; r.SW = R[rc - TT::RW - 1];
            const uint32_t node = (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
            float2 z = make_float2(0.f, 0.f);
            if (MODE == 2) z = a.xi49[(long long)y * g.nx + x];
            if (MODE == 3) z = stencil_xi<TT::HW>(H, TT::HN, lx, ly);
            float o[Q];
            collide_node<MODE, POLY, GF>(a, f, r, node, z, o);
            store9<T, float, GF>(static_cast<T*>(a.dst), g.plane, g, x, y, o);
        }
    }
}

// --- host side ----------------------------------------------------------------------

EncodeTiledFn tensor_map_encoder() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        const bool ok = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                            cudaSuccess && q == cudaDriverEntryPointSuccess;
        return ok ? (EncodeTiledFn)p : (EncodeTiledFn) nullptr;
    }();
    return fn;
}

// Tile shapes (TX x TY nodes, NT threads): 0 = 32x16/256, 1 = 32x32/256, 2 = 64x8/256,
// 3 = 64x16/512, 4 = 32x16/128.
static const int kTiles[5][3] = {{32, 16, 256}, {32, 32, 256}, {64, 8, 256}, {64, 16, 512}, {32, 16, 128}};

int tma_tile_count() { return 5; }

// The fastest shape per noise mode (0 off, 1 uncorrelated, 2 correlated, 3 correlated built
// in real space) and storage, measured on GB300 at 4096^2: FP32 off 32x32 (263 us),
// uncorrelated 32x32 (212.5 us against 214.1 for 64x16/512, alternating runs on one box),
// correlated 32x16 (235.0 us; 32x32 285, 64x16 240), real space 32x16 (334 us; 32x32 422);
// FP16 off 32x16/128 (153 us), uncorrelated 32x32 (220.1 us; the others 221-226),
// correlated 64x16 (245 us).
int tma_default_tile(int noise_mode, int fp16) {
    static const int best[2][5] = {{1, 1, 0, 0, 3}, {4, 1, 3, 0, 1}};
    const int m = noise_mode < 0 ? 0 : (noise_mode > 4 ? 4 : noise_mode);
    return best[fp16 ? 1 : 0][m];
}

// Tensor map over one population buffer: dims (pitch, ny + 2 GY, 9) of FP32, box
// (TX + 8, TY + 2, 1), zero fill outside.
bool make_pop_tensor_map(const void* buf, const Grid& g, int tile, int fp16, void* map_out) {
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn || tile < 0 || tile >= tma_tile_count()) return false;
    const cuuint64_t es = fp16 ? 2 : 4;
    const int xo = fp16 ? Elem<__half>::XO : Elem<float>::XO;
    cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * GY), (cuuint64_t)Q};
    cuuint64_t strides[2] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.plane * es};
    cuuint32_t box[3] = {(cuuint32_t)(kTiles[tile][0] + 2 * xo), (cuuint32_t)kTiles[tile][1] + 2, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map_out),
                    fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)buf, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t tensor_map_bytes() { return sizeof(CUtensorMap); }

template <int TX, int TY, int NT, int MODE, typename T, bool POLY = false>
static cudaError_t launch_cfg(const void* map, TmaArgs ta, cudaStream_t s) {
    using TT = TmaTile<TX, TY, T>;
    auto kern = step_tma_kernel<TX, TY, NT, MODE, T, POLY>;
    constexpr int smem = TT::SMEM_BYTES + (MODE == 3 ? TT::H_BYTES : 0);
    static GridCache cache;
    int grid_max = 0;
    cudaError_t e = resident_grid(kern, NT, smem, cache, &grid_max);
    if (e != cudaSuccess) return e;
    ta.ntx = (ta.a.g.nx + TX - 1) / TX;
    ta.nty = (ta.a.g.ny + TY - 1) / TY;
    const int ntiles = ta.ntx * ta.nty;
    const int grid = ntiles < grid_max ? ntiles : grid_max;
    kern<<<grid, NT, smem, s>>>(*reinterpret_cast<const CUtensorMap*>(map), ta);
    return cudaGetLastError();
}

template <int MODE, typename T>
static cudaError_t launch_mode(const void* map, const TmaArgs& ta, int tile, cudaStream_t s) {
    switch (tile) {
        case 1: return launch_cfg<32, 32, 256, MODE, T>(map, ta, s);
        case 2: return launch_cfg<64, 8, 256, MODE, T>(map, ta, s);
        case 3: return launch_cfg<64, 16, 512, MODE, T>(map, ta, s);
        case 4: return launch_cfg<32, 16, 128, MODE, T>(map, ta, s);
        default: return launch_cfg<32, 16, 256, MODE, T>(map, ta, s);
    }
}

template <typename T>
static cudaError_t launch_type(const void* map, const TmaArgs& ta, int noise_mode, int tile, cudaStream_t s) {
    switch (noise_mode) {
        case 0: return launch_mode<0, T>(map, ta, tile, s);
        case 1: return launch_mode<1, T>(map, ta, tile, s);
        case 3: return launch_mode<3, T>(map, ta, tile, s);
        case 4: return launch_mode<4, T>(map, ta, tile, s);
        default: return launch_mode<2, T>(map, ta, tile, s);
    }
}

// the double-well equation of state, FP32 storage: the default tile of each noise mode
// (tma_default_tile(noise_mode, 0); the caller encodes the tensor maps for it)
static cudaError_t launch_poly(const void* map, const TmaArgs& ta, int noise_mode, cudaStream_t s) {
    switch (noise_mode) {
        case 0: return launch_cfg<32, 32, 256, 0, float, true>(map, ta, s);
        case 1: return launch_cfg<64, 16, 512, 1, float, true>(map, ta, s);
        case 3: return launch_cfg<32, 16, 256, 3, float, true>(map, ta, s);
        case 4: return launch_cfg<64, 16, 512, 4, float, true>(map, ta, s);
        default: return launch_cfg<32, 16, 256, 2, float, true>(map, ta, s);
    }
}

cudaError_t launch_step_tma(const StepArgs& a, const void* src_map, int* err, int noise_mode, int tile, int fp16,
                            cudaStream_t s, bool poly) {
    TmaArgs ta;
    ta.a = a;
    ta.ntx = ta.nty = 0;
    ta.err = err;
    if (poly) return fp16 ? cudaErrorInvalidValue : launch_poly(src_map, ta, noise_mode, s);
    return fp16 ? launch_type<__half>(src_map, ta, noise_mode, tile, s)
                : launch_type<float>(src_map, ta, noise_mode, tile, s);
}

}  // namespace lbf
