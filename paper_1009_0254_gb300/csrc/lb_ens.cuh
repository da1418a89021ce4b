// lb_ens.cuh -- device pieces shared by the engines that step many independent lattices
// in one launch (batched ensembles, the request server): the per-lattice record, the
// register copy of it that the collision reads, and the collision of one staged tile.
#pragma once

#include "lb_collide.cuh"
#include "lb_internal.cuh"
#include "lb_tma.cuh"

#include <type_traits>

namespace lbf {

// Per-replica record (device).
struct RepRec {
    float rho0, cs2m, kappa, lb, ls, lq, le;
    float L44, L49, L94, L99, s5, s6, s7;
    float a44, b44, a49, b49, a99, b99;   // Xi(k) of the (4,9) block = a + b s(k) (correlated noise)
    int mode;                 // 0 no noise, 1 uncorrelated, 2 correlated (k-space), 3 correlated (real space)
    uint32_t k0, k1;          // Philox key = the replica's seed
    long long toff;           // time = K + toff
    float sL[3][4];           // real-space correlated noise: factors / 4 of Xi at k^2 = 0, 4, 16/3
};

// What collide_node needs for one tile of one replica, in registers (the engines step the
// linearised equation of state).
struct __align__(16) TileArgs {
    RoundKeys4 rk;            // the lattice's Philox round keys
    float rho0, cs2m, kappa, lb, ls, lq, le;
    float L44, L49, L94, L99, s5, s6, s7;
    uint32_t t_lo, t_hi;
};

// The same with the real-space correlated-noise factors: the record of the engines' step
// kernel variant that steps such lattices (the lean variant keeps the smaller record).
struct TileArgsRS : TileArgs {
    float sL[3][4];
};

template <bool RS>
using TileArgsOf = typename std::conditional<RS, TileArgsRS, TileArgs>::type;

// The record of one lattice as collide_node reads it, for its time t, written by one
// thread into the tile's shared record a; *mode = 0 without noise, 1 with uncorrelated
// noise, 2 with correlated noise (xi_4, xi_9 read from a field), 3 with correlated noise
// built in real space.
__device__ __forceinline__ void load_tile_args(const RepRec* rp, long long t, TileArgs* a, int* mode) {
    a->rho0 = __ldg(&rp->rho0); a->cs2m = __ldg(&rp->cs2m); a->kappa = __ldg(&rp->kappa);
    a->lb = __ldg(&rp->lb); a->ls = __ldg(&rp->ls); a->lq = __ldg(&rp->lq); a->le = __ldg(&rp->le);
    a->L44 = __ldg(&rp->L44); a->L49 = __ldg(&rp->L49); a->L94 = __ldg(&rp->L94); a->L99 = __ldg(&rp->L99);
    a->s5 = __ldg(&rp->s5); a->s6 = __ldg(&rp->s6); a->s7 = __ldg(&rp->s7);
    uint32_t k0 = __ldg(&rp->k0), k1 = __ldg(&rp->k1);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        a->rk.q[j] = make_uint4(k0, k1, k0 + 0x9E3779B9u, k1 + 0xBB67AE85u);
        k0 += 2u * 0x9E3779B9u;
        k1 += 2u * 0xBB67AE85u;
    }
    a->t_lo = (uint32_t)((unsigned long long)t & 0xffffffffu);
    a->t_hi = (uint32_t)((unsigned long long)t >> 32);
    *mode = __ldg(&rp->mode);
}

// The real-space correlated-noise factors of a record (only for its lattices with that
// mode: the record load sits on the tile's critical path).
__device__ __forceinline__ void load_stencil_args(const RepRec* rp, TileArgsRS* a) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) a->sL[j][q] = __ldg(&rp->sL[j][q]);
}

// Pulls the nine deviations of this thread's nodes of the staged tile S into registers
// (fr) and writes the density deviation of the tile and of its one-node ring (from the
// halo) into R.  After a CTA barrier the stage is no longer read.  The ring goes to the
// last threads (the first loads the tile's record and issues the refill) unless the
// launch may hold real-space correlated noise (RS), whose halo contributions the last
// threads form.
template <int TX, int TY, int NT, bool RS>
__device__ __forceinline__ void tile_pull(const float* S, float* R, float (&fr)[TX * TY / NT][Q]) {
    using TT = TmaTile<TX, TY, float>;
    static_assert((TX * TY) % NT == 0, "tile must be a multiple of the block");
#pragma unroll
    for (int it = 0; it < TX * TY / NT; ++it) {
        const int q = threadIdx.x + it * NT;
        const int ly = q / TX, lx = q - ly * TX;
        load9_ps<TT::PS>(S, (ly + 1) * TT::BW + lx + TT::XO, fr[it]);
        R[(ly + 1) * TT::RW + lx + 1] = drho_of(fr[it]);
    }
    // the ring: rows 0 and TY + 1 (TX + 2 each), then columns 0 and TX + 1
    constexpr int NB = 2 * (TX + 2) + 2 * TY;
    for (int j = RS ? (int)threadIdx.x : NT - 1 - (int)threadIdx.x; j < NB; j += NT) {
        int rx, ry;
        if (j < TX + 2) { rx = j; ry = 0; }
        else if (j < 2 * (TX + 2)) { rx = j - (TX + 2); ry = TY + 1; }
        else { const int u = j - 2 * (TX + 2); ry = 1 + (u >> 1); rx = (u & 1) ? TX + 1 : 0; }
        float h[Q];
        load9_ps<TT::PS>(S, ry * TT::BW + rx + TT::XO - 1, h);
        R[ry * TT::RW + rx] = drho_of(h);
    }
}

// Collide and stream the TX x TY nodes of one tile from the pulled deviations fr and the
// density tile R (with its one-node ring).  The record a is the tile's lattice, held in
// shared memory by the callers (registers are taken by fr).
template <int MODE, int TX, int TY, int NT>
__device__ __forceinline__ void tile_nodes(const TileArgs& a, const float (&fr)[TX * TY / NT][Q], const float* R,
                                           const Grid& g, int x0, int y0, float* dst,
                                           const float2* __restrict__ xi49, const float2* Hs = nullptr) {
    using TT = TmaTile<TX, TY, float>;
#pragma unroll
    for (int it = 0; it < TX * TY / NT; ++it) {
        const int q = threadIdx.x + it * NT;
        const int ly = q / TX, lx = q - ly * TX;
        const int x = x0 + lx, y = y0 + ly;
        if (x >= g.nx || y >= g.ny) continue;
        const int rc = (ly + 1) * TT::RW + lx + 1;
        Nbr r;
        r.C = R[rc];
        r.E = R[rc + 1]; r.W = R[rc - 1];
        r.N = R[rc + TT::RW]; r.S = R[rc - TT::RW];
        r.NE = R[rc + TT::RW + 1]; r.NW = R[rc + TT::RW - 1];
        r.SE = R[rc - TT::RW + 1]; r.SW = R[rc - TT::RW - 1];
        const uint32_t node = (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
        float2 z = make_float2(0.f, 0.f);
        if (MODE == 2) z = xi49[(long long)y * g.nx + x];
        if (MODE == 3) z = stencil_xi<TT::HW>(Hs, TT::HN, lx, ly);
        float o[Q];
        collide_node<MODE>(a, fr[it], r, node, z, o);
        store9(dst, g.plane, g, x, y, o);
    }
}

// Real-space correlated noise of a staged tile whose lattice uses it: the 2 x 2-box
// contributions of the tile's nodes and of its halo, written into the memory of the stage
// just consumed (FP32 stages hold them; the caller refills that stage after the collision).
template <int TX, int TY, int NT>
__device__ __forceinline__ void tile_stencil(const TileArgsRS& a, float2* Hs, const Grid& g, int x0, int y0) {
    using TT = TmaTile<TX, TY, float>;
    static_assert(TT::H_IN_STAGE, "the noise contributions must fit in a stage");
#pragma unroll 1
    for (int it = 0; it < TX * TY / NT; ++it) {
        const int q = threadIdx.x + it * NT;
        const int ly = q / TX, lx = q - ly * TX;
        const int x = x0 + lx, y = y0 + ly;
        if (x < g.nx && y < g.ny)
            stencil_store<TT::HW>(a, Hs, TT::HN, lx, ly, (uint32_t)y * (uint32_t)g.nx + (uint32_t)x);
    }
    stencil_halo<TX, TY, TT::HW>(a, Hs, TT::HN, x0, y0, g.nx, g.ny, threadIdx.x, NT);
}

// host: fills the parameter fields of a record (defined in lb_batch.cu)
void fill_rep_record(double rho0, double cs2, double kT, double kappa, double tau_s, double tau_b,
                     double tau_ghost, int noise_mode, RepRec* rec);

}  // namespace lbf
