// lb3d.cu -- the fused fluctuating step on the D3Q19 and D3Q27 lattices for sm_103a and the
// C ABI of lbfluct3d.h.
//
// One launch performs one time step on every node (collision of lb3_collide.cuh or
// lb27_collide.cuh, then streaming in pull form: f_i(r, t) = f*_i(r - c_i, t - 1)).  A CTA
// owns a TX x TY tile of the (x, y) plane and marches over a run of z planes.  The pulled
// populations of each plane, for the tile and its one-node ring, are staged in shared
// memory by asynchronous copies (three rotating slots: the plane being collided, the plane
// whose densities are summed, and the plane in flight), so the loads of plane z+2 overlap
// the collision of plane z.  With two slots (D3Q27's default: its smaller shared-memory
// footprint fits four CTAs per SM instead of three) a plane's own populations move to
// registers when its densities are summed.  The densities of planes z-1, z, z+1 sit in three more rotating
// slots; the collision reads its own node's populations and its 3x3x3 density neighbourhood
// from shared memory.  Every population is read once from DRAM (the ring's re-reads hit L2)
// and written once: 2 Q sizeof(storage) bytes per node.
//
// A plain D3Q19 kernel (density summed from direct loads, the collision pulling again) is
// kept as a cross-check (LBFLUCT3_KERNEL=plain).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "lb27_collide.cuh"
#include "lb3_collide.cuh"
#include "lb_internal.cuh"
#include "lbfluct3d.h"

namespace lbf3 {

constexpr double SIGMA_S2 = 1.0 / 3.0;
constexpr int QMAX = 27;

// velocity components in {-1, 0, 1} packed two bits each: c = ((P >> 2i) & 3) - 1
constexpr unsigned long long pack3(const int (&v)[19]) {
    unsigned long long p = 0;
    for (int i = 0; i < 19; ++i) p |= (unsigned long long)(v[i] + 1) << (2 * i);
    return p;
}

// D3Q19: the velocity order of lb3_collide.cuh; noise tags 4, 5
struct Lat19 {
    static constexpr int Q = 19, TX = 32, TY = 8;
    static constexpr uint32_t TAG0 = 4;
    static constexpr int CXv[19] = {0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
    static constexpr int CYv[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 0, 0, 0, 0};
    static constexpr int CZv[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1};
    static constexpr unsigned long long PX = pack3(CXv), PY = pack3(CYv), PZ = pack3(CZv);
    __host__ __device__ static constexpr int c(int i, int k) {
        return (int)(((k == 0 ? PX : (k == 1 ? PY : PZ)) >> (2 * i)) & 3ULL) - 1;
    }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

// D3Q27: i = 9 ix + 3 iy + iz, components (0, 1, -1); noise tags 6, 7, 8
struct Lat27 {
    static constexpr int Q = 27, TX = 32, TY = 4;
    static constexpr uint32_t TAG0 = 6;
    __host__ __device__ static constexpr int v(int a) { return a == 0 ? 0 : (a == 1 ? 1 : -1); }
    __host__ __device__ static constexpr int c(int i, int k) {
        return v(k == 0 ? i / 9 : (k == 1 ? (i / 3) % 3 : i % 3));
    }
    __host__ __device__ static constexpr double w1(int a) { return a == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double w(int i) { return w1(i / 9) * w1((i / 3) % 3) * w1(i % 3); }
};

// The D3Q27 modes whose noise is coupled (the Cholesky factor's dense 7 x 7 block, in mode
// order): p_2z, p_2y, p_2y p_2z, p_2x, p_2x p_2z, p_2x p_2y, p_2x p_2y p_2z.
constexpr int COUPLED27[7] = {2, 6, 8, 18, 20, 24, 26};
__host__ __device__ constexpr int coupled27(int r) {
    return r == 0 ? 2 : (r == 1 ? 6 : (r == 2 ? 8 : (r == 3 ? 18 : (r == 4 ? 20 : (r == 5 ? 24 : 26)))));
}

template <typename R>
struct Step3Args {
    const R* __restrict__ src;    // post-collision deviations at t-1, Q planes of P nodes
    R* __restrict__ dst;
    int nx, ny, nz, zc;           // zc: planes per CTA
    long long P;                  // nodes per population plane
    Coef3<R> co;
    R sc[QMAX];                   // sqrt(Xi_kk) of the modes with a diagonal factor
    R Lc[28];                     // the coupled block's Cholesky factor: D3Q19 (L44, L16_4, L16_16);
                                  // D3Q27 the 7 x 7 lower triangle, row-major
    R Lrs[9];                     // D3Q19 correlated noise: Cholesky factors (L11, L21, L22) of the
                                  // (4,16) block of Xi at s = 0, 4, 16/3
    uint32_t t_lo, t_hi;
    lbf::RoundKeys rk;
};

// D3Q19 noise: tag 4 -> nu_4..nu_11, tag 5 -> nu_12..nu_18
template <typename R>
__device__ __forceinline__ void normals19(const Step3Args<R>& a, uint32_t node, R xi[Q3]) {
    const uint4 ra = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, Lat19::TAG0), a.rk);
    const uint4 rb = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, Lat19::TAG0 + 1), a.rk);
    R n4, n16, spare;
    lbf::gauss_word(ra.x, &n4, &xi[5]);
    lbf::gauss_word(ra.y, &xi[6], &xi[7]);
    lbf::gauss_word(ra.z, &xi[8], &xi[9]);
    lbf::gauss_word(ra.w, &xi[10], &xi[11]);
    lbf::gauss_word(rb.x, &xi[12], &xi[13]);
    lbf::gauss_word(rb.y, &xi[14], &xi[15]);
    lbf::gauss_word(rb.z, &n16, &xi[17]);
    lbf::gauss_word(rb.w, &xi[18], &spare);
    (void)spare;
#pragma unroll
    for (int q = 5; q < Q3; ++q) xi[q] *= a.sc[q];
    xi[4] = a.Lc[0] * n4;
    xi[16] = a.Lc[1] * n4 + a.Lc[2] * n16;
}

// position of mode k among the non-conserved D3Q27 modes (conserved: 0, 1, 3, 9)
__host__ __device__ constexpr int nc27(int k) { return k - (k > 0) - (k > 1) - (k > 3) - (k > 9); }

// D3Q27 noise: tags 6, 7, 8 give 24 normals; normal n goes to the n-th non-conserved mode
template <typename R>
__device__ __forceinline__ void normals27(const Step3Args<R>& a, uint32_t node, R xi[Q27]) {
    R nu[24];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const uint4 r = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, Lat27::TAG0 + d), a.rk);
        lbf::gauss_word(r.x, &nu[8 * d + 0], &nu[8 * d + 1]);
        lbf::gauss_word(r.y, &nu[8 * d + 2], &nu[8 * d + 3]);
        lbf::gauss_word(r.z, &nu[8 * d + 4], &nu[8 * d + 5]);
        lbf::gauss_word(r.w, &nu[8 * d + 6], &nu[8 * d + 7]);
    }
#pragma unroll
    for (int k = 0; k < Q27; ++k)
        xi[k] = (k == 0 || k == 1 || k == 3 || k == 9) ? R(0) : a.sc[k] * nu[nc27(k)];
#pragma unroll
    for (int r = 0; r < 7; ++r) {
        R s = R(0);
#pragma unroll
        for (int q = 0; q <= r; ++q) s += a.Lc[r * (r + 1) / 2 + q] * nu[nc27(coupled27(q))];
        xi[coupled27(r)] = s;
    }
}

__device__ __forceinline__ int wrap_lo(int v, int n) { return v < 0 ? v + n : v; }
__device__ __forceinline__ int wrap_hi(int v, int n) { return v >= n ? v - n : v; }

// asynchronous global -> shared copy of one element (4 or 8 bytes), cached in L1
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// density deviation of one node's pulled deviations, one fixed summation order
template <typename LAT, typename R>
__device__ __forceinline__ R drho_of(const R* f) {
    if constexpr (LAT::Q == 19) {
        return drho19(f);
    } else {
        R s = f[0];
#pragma unroll
        for (int i = 1; i < Q27; i += 2) s += (i + 1 < Q27) ? (f[i] + f[i + 1]) : f[i];
        return s;
    }
}

// D3Q19 correlated noise: the tags of the two draws of the eight corner fields
constexpr uint32_t TAG_RS0 = 10;

// The staged step kernel: one CTA per TX x TY tile and run of zc planes.  With correlated
// noise (MODE 3) it also holds the 2x2x2-box contributions: for the tile plus its left column
// and bottom row, the in-plane half (four 2-vectors) of the current plane and the upward half
// of the current and the previous plane.
template <typename LAT, typename R, int SLOTS, int MODE>
constexpr int staged_smem_bytes() {
    return ((SLOTS * LAT::Q + 3) * (LAT::TX + 2) * (LAT::TY + 2) +
            (MODE == 3 ? 24 * (LAT::TX + 1) * (LAT::TY + 1) : 0)) * (int)sizeof(R);
}

// resident CTAs per SM the register budget is sized for: as many as the shared memory admits
// (227 KB per SM, 1 KB reserved per CTA), at most 2048 threads
template <typename LAT, typename R, int SLOTS, int MODE>
constexpr int staged_min_blocks() {
    constexpr int by_smem = (227 * 1024) / (staged_smem_bytes<LAT, R, SLOTS, MODE>() + 1024);
    constexpr int by_threads = 2048 / (LAT::TX * LAT::TY);
    return by_smem < 1 ? 1 : (by_smem < by_threads ? by_smem : by_threads);
}

template <typename LAT, typename R, int MODE, typename I, int SLOTS>
__global__ void __launch_bounds__(LAT::TX * LAT::TY, staged_min_blocks<LAT, R, SLOTS, MODE>())
    step3_staged_kernel(const Step3Args<R> a) {
    constexpr int Q = LAT::Q, TX = LAT::TX, TY = LAT::TY;
    constexpr int RX = TX + 2, RY = TY + 2, RN = RX * RY, NT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem3[];
    R* raw = reinterpret_cast<R*>(smem3);                   // [SLOTS][Q][RN] pulled populations
    R* rs = raw + SLOTS * Q * RN;                           // [3][RN] density deviations
    constexpr int HW = TX + 1, HN = HW * (TY + 1);
    R* Hin = rs + 3 * RN;                                   // MODE 3: [8][HN] in-plane half
    R* Hup = Hin + 8 * HN;                                  // MODE 3: [2][8][HN] upward half
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long P = a.P, nxy = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, nz);
    const int tid = threadIdx.x;
    const R* __restrict__ src = a.src;
    // offsets in I: 32-bit when all Q planes fit in 2^32 elements, else 64-bit
    const I PI = (I)P;

    // The tile-and-ring positions a thread stages are the same on every plane: their validity
    // and the nine in-plane offsets (x - cx) + (y - cy) nx, indexed (1 - cy) 3 + (1 - cx), are
    // formed once.
    constexpr int KP = (RN + NT - 1) / NT;
    I yx[KP][9];
    bool valid[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int q = tid + k * NT;
        const int ly = q / RX, lx = q - ly * RX;
        int gx = x0 + lx - 1, gy = y0 + ly - 1;
        valid[k] = q < RN && gx <= nx && gy <= ny;      // others are never read by a node
        gx = wrap_hi(wrap_lo(gx, nx), nx);
        gy = wrap_hi(wrap_lo(gy, ny), ny);
        const I Xo[3] = {(I)(gx == 0 ? nx - 1 : gx - 1), (I)gx, (I)(gx == nx - 1 ? 0 : gx + 1)};
        const I Yo[3] = {(I)(gy == 0 ? ny - 1 : gy - 1) * (I)nx, (I)gy * (I)nx,
                         (I)(gy == ny - 1 ? 0 : gy + 1) * (I)nx};
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) yx[k][3 * b + c] = Yo[b] + Xo[c];
    }

    // issue the pulled populations of plane zz (an integer in [-1, nz]) into raw slot k
    auto issue = [&](int zz, int slot_k) {
        const int zc = wrap_hi(wrap_lo(zz, nz), nz);
        // plane offsets of z - cz, indexed by 1 - cz
        const I Zo[3] = {(I)(zc == 0 ? nz - 1 : zc - 1) * (I)nxy, (I)zc * (I)nxy,
                         (I)(zc == nz - 1 ? 0 : zc + 1) * (I)nxy};
        R* slot = raw + slot_k * Q * RN;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            if (!valid[k]) continue;
            const int q = tid + k * NT;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const I off = (I)i * PI + Zo[1 - LAT::c(i, 2)] + yx[k][3 * (1 - LAT::c(i, 1)) + (1 - LAT::c(i, 0))];
                cp_async_elem<sizeof(R)>(slot + i * RN + q, src + off);
            }
        }
        cp_async_commit();
    };
    // density deviations of the plane in raw slot slot_k into density slot dk; positions run
    // from the last thread down, so the positions beyond the block's width fall on other
    // threads than the extra copies of issue()
    auto density = [&](int slot_k, int dk) {
        const R* slot = raw + slot_k * Q * RN;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int q = (NT - 1 - tid) + k * NT;
            if (q >= RN) continue;
            const int ly = q / RX, lx = q - ly * RX;
            R v = R(0);
            if (x0 + lx - 1 <= nx && y0 + ly - 1 <= ny) {
                R f[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) f[i] = slot[i * RN + q];
                v = drho_of<LAT>(f);
            }
            rs[dk * RN + q] = v;
        }
    };

    const int lx = tid % TX, ly = tid / TX;
    const int x = x0 + lx, y = y0 + ly;
    const bool own = x < nx && y < ny;
    const int qc = (ly + 1) * RX + lx + 1;

    // MODE 3: the eight white 2-vectors nu_w of every position of plane zz (tile, left column,
    // bottom row), times the factor of their corner (w = 4 ia + 2 ib + ic, sign -1 for a set
    // bit: k = pi), combined by a Walsh-Hadamard transform into h_m = (1/8) sum_w
    // (-1)^{popcount(w & m)} L_w nu_w, m = 4 dx + 2 dy + dz: the in-plane half (dz = 0) into Hin
    // when keep_in, the upward half (dz = 1) into buffer ub
    auto stencil_plane = [&](int zz, bool keep_in, int ub) {
        const int zc = wrap_hi(wrap_lo(zz, nz), nz);
        for (int p = NT - 1 - tid; p < HN; p += NT) {       // extra positions on the last threads
            const int hy = p / HW - 1, hx = p - (hy + 1) * HW - 1;
            int gx = x0 + hx, gy = y0 + hy;
            if (gx >= nx || gy >= ny) continue;         // never read by a node of the lattice
            gx = wrap_lo(gx, nx);
            gy = wrap_lo(gy, ny);
            const uint32_t node = ((uint32_t)zc * (uint32_t)ny + (uint32_t)gy) * (uint32_t)nx + (uint32_t)gx;
            const uint4 r0 = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_RS0), a.rk);
            const uint4 r1 = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, TAG_RS0 + 1), a.rk);
            const uint32_t wd[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            R vx[8], vy[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                R n0, n1;
                lbf::gauss_word(wd[w], &n0, &n1);
                const int pc = (w & 1) + ((w >> 1) & 1) + ((w >> 2) & 1);      // components at pi
                const int cls = pc == 0 ? 0 : (pc == 2 ? 2 : 1);             // s = 0, 16/3, 4
                vx[w] = a.Lrs[3 * cls] * n0;
                vy[w] = a.Lrs[3 * cls + 1] * n0 + a.Lrs[3 * cls + 2] * n1;
            }
#pragma unroll
            for (int b = 1; b < 8; b <<= 1)
#pragma unroll
                for (int w = 0; w < 8; ++w)
                    if (!(w & b)) {
                        const R ax = vx[w], ay = vy[w], bx = vx[w | b], by = vy[w | b];
                        vx[w] = ax + bx; vy[w] = ay + by;
                        vx[w | b] = ax - bx; vy[w | b] = ay - by;
                    }
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                R* dst = (m & 1) ? Hup + ub * 8 * HN : Hin;
                if (!(m & 1) && !keep_in) continue;
                const int j = m >> 1;
                dst[(2 * j) * HN + p] = R(0.125) * vx[m];
                dst[(2 * j + 1) * HN + p] = R(0.125) * vy[m];
            }
        }
    };

    // the collision of plane z from its pulled values f and density slots of z, z-1, z+1
    // (hb: the buffer of the previous plane's upward noise contributions, MODE 3)
    auto collide_plane = [&](int z, const R (&f)[Q], int k0, int km, int kp, int hb) {
        const R* d0 = rs + k0 * RN + qc;
        const R* dm = rs + km * RN + qc;
        const R* dp = rs + kp * RN + qc;
        R xi[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) xi[q] = R(0);
        const I node = (I)z * (I)nxy + (I)y * (I)nx + (I)x;
        R o[Q];
        if constexpr (Q == 19) {
            Rho3<R> r;
            r.c = d0[0];
            r.xp = d0[1]; r.xm = d0[-1];
            r.yp = d0[RX]; r.ym = d0[-RX];
            r.zp = dp[0]; r.zm = dm[0];
            r.ap = d0[RX + 1]; r.am = d0[-RX - 1];         // (1,1,0)
            r.bp = d0[-RX + 1]; r.bm = d0[RX - 1];         // (1,-1,0)
            r.cp = dp[RX]; r.cm = dm[-RX];                 // (0,1,1)
            r.dp = dm[RX]; r.dm = dp[-RX];                 // (0,1,-1)
            r.ep = dp[1]; r.em = dm[-1];                   // (1,0,1)
            r.fp = dp[-1]; r.fm = dm[1];                   // (-1,0,1)
            if (MODE == 1 || MODE == 3) normals19(a, (uint32_t)node, xi);
            if constexpr (MODE == 3) {
                // (xi_4, xi_16) = sum over the box: h of r - (dx, dy, 0) from this plane and of
                // r - (dx, dy, 1) from the previous one
                R s4 = R(0), s16 = R(0);
                const R* hu = Hup + hb * 8 * HN;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int q = (ly - (j & 1) + 1) * HW + (lx - (j >> 1) + 1);
                    s4 += Hin[(2 * j) * HN + q] + hu[(2 * j) * HN + q];
                    s16 += Hin[(2 * j + 1) * HN + q] + hu[(2 * j + 1) * HN + q];
                }
                xi[4] = s4;
                xi[16] = s16;
            }
            collide19(a.co, f, r, xi, o);
        } else {
            // nb[i] = rho(r + c_i)
            R nb[Q27];
#pragma unroll
            for (int i = 0; i < Q27; ++i) {
                const int cz = LAT::c(i, 2);
                const R* pl = cz == 0 ? d0 : (cz > 0 ? dp : dm);
                nb[i] = pl[LAT::c(i, 1) * RX + LAT::c(i, 0)];
            }
            if (MODE == 1) normals27(a, (uint32_t)node, xi);
            collide27(a.co, f, nb, xi, o);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) a.dst[(I)i * PI + node] = o[i];
    };

    if constexpr (SLOTS == 3) {
        // planes z0-1, z0 -> slots 0, 1; plane z0+1 -> slot 2 (in flight); density slots alike
        issue(z0 - 1, 0);
        issue(z0, 1);
        cp_async_wait_all();
        __syncthreads();
        density(0, 0);
        density(1, 1);
        if constexpr (MODE == 3) stencil_plane(z0 - 1, false, 0);
        issue(z0 + 1, 2);
        for (int z = z0; z < z1; ++z) {
            const int k0 = (z - z0 + 1) % 3, km = (k0 + 2) % 3, kp = (k0 + 1) % 3;   // slots of z, z-1, z+1
            cp_async_wait_all();
            __syncthreads();
            density(kp, kp);
            if constexpr (MODE == 3) stencil_plane(z, true, (z - z0 + 1) & 1);
            if (z + 1 < z1) issue(z + 2, km);          // plane z-1's slot is free
            __syncthreads();
            if (!own) continue;
            const R* sl = raw + k0 * Q * RN;
            R f[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = sl[i * RN + qc];
            collide_plane(z, f, k0, km, kp, (z - z0) & 1);
        }
    } else {
        // two raw slots: a plane's own pulled values move to registers when its densities are
        // summed, which frees its slot for the plane after next
        R fcur[Q], fnext[Q];
        auto take = [&](int k, R (&f)[Q]) {
            const R* sl = raw + k * Q * RN;
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = own ? sl[i * RN + qc] : R(0);
        };
        issue(z0 - 1, 0);
        issue(z0, 1);
        cp_async_wait_all();
        __syncthreads();
        density(0, 0);                 // plane z0-1 -> density slot 0
        density(1, 1);                 // plane z0 -> density slot 1
        take(1, fcur);
        if constexpr (MODE == 3) stencil_plane(z0 - 1, false, 0);
        __syncthreads();
        issue(z0 + 1, 0);              // raw slot of plane p: (p - z0 + 1) % 2
        for (int z = z0; z < z1; ++z) {
            const int k0 = (z - z0 + 1) % 3, km = (k0 + 2) % 3, kp = (k0 + 1) % 3;
            const int rp = (z - z0) & 1;             // raw slot of plane z+1
            cp_async_wait_all();
            __syncthreads();
            if (z + 1 < z1) issue(z + 2, rp ^ 1);    // the slot of plane z, already in registers
            density(rp, kp);
            take(rp, fnext);
            if constexpr (MODE == 3) stencil_plane(z, true, (z - z0 + 1) & 1);
            __syncthreads();
            if (own) collide_plane(z, fcur, k0, km, kp, (z - z0) & 1);
#pragma unroll
            for (int i = 0; i < Q; ++i) fcur[i] = fnext[i];
        }
    }
    cp_async_wait_all();
}

// ---- the plain D3Q19 kernel (cross-check) -----------------------------------------------

// the 19 pulled deviations of node (x, y, z): f_i = src_i(r - c_i)
template <typename R>
__device__ __forceinline__ void pull19(const R* __restrict__ s, long long P, int x, int xm, int xp, long long ym,
                                       long long y0, long long yp, long long zm, long long z0, long long zp,
                                       R f[Q3]) {
    f[0] = s[z0 + y0 + x];
    f[1] = s[P + z0 + y0 + xm];
    f[2] = s[2 * P + z0 + y0 + xp];
    f[3] = s[3 * P + z0 + ym + x];
    f[4] = s[4 * P + z0 + yp + x];
    f[5] = s[5 * P + zm + y0 + x];
    f[6] = s[6 * P + zp + y0 + x];
    f[7] = s[7 * P + z0 + ym + xm];
    f[8] = s[8 * P + z0 + yp + xm];
    f[9] = s[9 * P + z0 + ym + xp];
    f[10] = s[10 * P + z0 + yp + xp];
    f[11] = s[11 * P + zm + ym + x];
    f[12] = s[12 * P + zp + ym + x];
    f[13] = s[13 * P + zm + yp + x];
    f[14] = s[14 * P + zp + yp + x];
    f[15] = s[15 * P + zm + y0 + xm];
    f[16] = s[16 * P + zm + y0 + xp];
    f[17] = s[17 * P + zp + y0 + xm];
    f[18] = s[18 * P + zp + y0 + xp];
}

template <typename R, int MODE, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) step3_kernel(const Step3Args<R> a) {
    constexpr int RX = TX + 2, RY = TY + 2, NT = TX * TY;
    __shared__ R rs[3][RY][RX];
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long P = a.P, nxy = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, nz);
    const int tid = threadIdx.x;
    const R* __restrict__ src = a.src;

    auto density = [&](int zz, int slot) {
        const int zc = wrap_hi(wrap_lo(zz, nz), nz);
        const long long Z0 = zc * nxy;
        const long long Zm = (zc == 0 ? nz - 1 : zc - 1) * nxy, Zp = (zc == nz - 1 ? 0 : zc + 1) * nxy;
        for (int q = tid; q < RX * RY; q += NT) {
            const int ly = q / RX, lx = q - ly * RX;
            int gx = x0 + lx - 1, gy = y0 + ly - 1;
            R v = R(0);
            if (gx <= nx && gy <= ny) {
                gx = wrap_hi(wrap_lo(gx, nx), nx);
                gy = wrap_hi(wrap_lo(gy, ny), ny);
                const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
                const long long Y0 = (long long)gy * nx;
                const long long Ym = (long long)(gy == 0 ? ny - 1 : gy - 1) * nx;
                const long long Yp = (long long)(gy == ny - 1 ? 0 : gy + 1) * nx;
                R f[Q3];
                pull19(src, P, gx, xm, xp, Ym, Y0, Yp, Zm, Z0, Zp, f);
                v = drho19(f);
            }
            rs[slot][ly][lx] = v;
        }
    };

    density(z0 - 1, 0);
    density(z0, 1);
    const int lx = tid % TX, ly = tid / TX;
    const int x = x0 + lx, y = y0 + ly;
    const bool own = x < nx && y < ny;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const long long Y0 = (long long)y * nx;
    const long long Ym = (long long)(y == 0 ? ny - 1 : y - 1) * nx;
    const long long Yp = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
    for (int z = z0; z < z1; ++z) {
        const int s0 = (z - z0 + 1) % 3, sm = (s0 + 2) % 3, sp = (s0 + 1) % 3;
        density(z + 1, sp);
        __syncthreads();
        if (own) {
            const long long Z0 = (long long)z * nxy;
            const long long Zm = (long long)(z == 0 ? nz - 1 : z - 1) * nxy;
            const long long Zp = (long long)(z == nz - 1 ? 0 : z + 1) * nxy;
            R f[Q3];
            pull19(src, P, x, xm, xp, Ym, Y0, Yp, Zm, Z0, Zp, f);
            const int cx = lx + 1, cy = ly + 1;
            Rho3<R> r;
            r.c = rs[s0][cy][cx];
            r.xp = rs[s0][cy][cx + 1]; r.xm = rs[s0][cy][cx - 1];
            r.yp = rs[s0][cy + 1][cx]; r.ym = rs[s0][cy - 1][cx];
            r.zp = rs[sp][cy][cx]; r.zm = rs[sm][cy][cx];
            r.ap = rs[s0][cy + 1][cx + 1]; r.am = rs[s0][cy - 1][cx - 1];
            r.bp = rs[s0][cy - 1][cx + 1]; r.bm = rs[s0][cy + 1][cx - 1];
            r.cp = rs[sp][cy + 1][cx]; r.cm = rs[sm][cy - 1][cx];
            r.dp = rs[sm][cy + 1][cx]; r.dm = rs[sp][cy - 1][cx];
            r.ep = rs[sp][cy][cx + 1]; r.em = rs[sm][cy][cx - 1];
            r.fp = rs[sp][cy][cx - 1]; r.fm = rs[sm][cy][cx + 1];
            R xi[Q3];
#pragma unroll
            for (int q = 0; q < Q3; ++q) xi[q] = R(0);
            const long long node = Z0 + Y0 + x;
            if (MODE == 1) normals19(a, (uint32_t)node, xi);
            R o[Q3];
            collide19(a.co, f, r, xi, o);
            R* __restrict__ d = a.dst + node;
#pragma unroll
            for (int i = 0; i < Q3; ++i) d[i * P] = o[i];
        }
        __syncthreads();
    }
}

template <typename LAT, typename R, int MODE, typename I, int SLOTS>
static cudaError_t launch_staged(const Step3Args<R>& a, dim3 grid, cudaStream_t s) {
    constexpr int smem = staged_smem_bytes<LAT, R, SLOTS, MODE>();
    // the shared-memory limit is a per-device attribute of the function: set it once per
    // device (a repeated set from a concurrent first launch is harmless)
    static std::atomic<unsigned> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned bit = 1u << (dev & 31);
    if (!(done.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(step3_staged_kernel<LAT, R, MODE, I, SLOTS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        done.fetch_or(bit, std::memory_order_release);
    }
    step3_staged_kernel<LAT, R, MODE, I, SLOTS><<<grid, LAT::TX * LAT::TY, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename LAT, typename R, int MODE>
static cudaError_t launch3(const Step3Args<R>& a, dim3 grid, bool plain, int slots, cudaStream_t s) {
    if constexpr (LAT::Q == 19) {
        if (plain) {
            step3_kernel<R, MODE, 32, 8><<<grid, 256, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    const bool narrow = (unsigned long long)a.P * LAT::Q < (1ULL << 32);
    if (slots == 2)
        return narrow ? launch_staged<LAT, R, MODE, uint32_t, 2>(a, grid, s)
                      : launch_staged<LAT, R, MODE, unsigned long long, 2>(a, grid, s);
    return narrow ? launch_staged<LAT, R, MODE, uint32_t, 3>(a, grid, s)
                  : launch_staged<LAT, R, MODE, unsigned long long, 3>(a, grid, s);
}

// ---- host-side theory --------------------------------------------------------------------

static double w_of(int lattice, int i) { return lattice == 19 ? Lat19::w(i) : Lat27::w(i); }
static int c_of(int lattice, int i, int k) { return lattice == 19 ? Lat19::c(i, k) : Lat27::c(i, k); }

// rest populations: w_i 3 cs2 rho0 on the moving velocities, the remainder at rest
static void rest_pops(int lattice, double rho0, double cs2, double* fbar) {
    double moving = 0.0;
    for (int i = 1; i < lattice; ++i) {
        fbar[i] = w_of(lattice, i) * 3.0 * cs2 * rho0;
        moving += fbar[i];
    }
    fbar[0] = rho0 - moving;
}

static double norm19(int a) {
    static const double N[Q3] = {1, 1.0 / 3, 1.0 / 3, 1.0 / 3, 2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                 2.0 / 3, 2.0 / 3, 2.0 / 3, 2.0 / 9, 2.0 / 9, 2.0 / 9, 2.0, 4.0 / 3, 4.0 / 9};
    return N[a];
}

// D3Q19 Xi(0) in closed form: in the variables y4 = m4 - d rho, y16 = m16 + d rho
// (d = 3 cs2 - 1) the linearised collision is diagonal and the equal-time covariances of the
// ansatz <df_i df_j> = (S/rho0) fbar_i delta_ij (S = rho0 kT / cs2) are rho0 kT (5 - 9 cs2),
// 9 rho0 kT (1 - cs2), 3 rho0 kT (3 cs2 - 1) for (y4, y4), (y16, y16), (y4, y16) and
// N_a rho0 kT / sigma_s^2 for the other non-conserved modes; stationarity under
// m -> (1 + lambda) m + xi gives the entries below.
static void xi_zero19(double rho0, double cs2, double kT, double lb, double ls, double lg, double* X) {
    for (int k = 0; k < Q3 * Q3; ++k) X[k] = 0.0;
    auto til = [](double l) { return l * (2.0 + l); };
    for (int a = 5; a < Q3; ++a) {
        const double l = a <= 9 ? ls : lg;
        X[a * Q3 + a] = -(rho0 * kT / SIGMA_S2) * norm19(a) * til(l);
    }
    X[4 * Q3 + 4] = -rho0 * kT * (5.0 - 9.0 * cs2) * til(lb);
    X[16 * Q3 + 16] = -9.0 * rho0 * kT * (1.0 - cs2) * til(lg);
    X[4 * Q3 + 16] = X[16 * Q3 + 4] = -3.0 * rho0 * kT * (3.0 * cs2 - 1.0) * (lb + lg + lb * lg);
}

// D3Q27 Xi(0).  The rest populations are fbar_i = 3 cs2 rho0 w_i + rho0 (1 - 3 cs2) delta_i0,
// so the ansatz covariance is the rank-one update G = S [3 cs2 diag(N) + (1 - 3 cs2) t0 t0^T]
// (t0: the modes at c = 0, S = rho0 kT / cs2).  With y = (I - J) m (J the density
// dependence of the equilibrium at rest) the ansatz makes y uncorrelated with rho, so the
// fluctuation-dissipation relation of Eq. (noise-matrix-k0) becomes
// Xi = -(Y Lambda^T + Lambda Y + Lambda Y Lambda^T) with Y = (I - J) G (I - J)^T.
static void xi_zero27(double rho0, double cs2, double kT, double lb, double ls, double lg, double* X) {
    constexpr int Q = Q27;
    const double n1[3] = {1.0, 1.0 / 3.0, 2.0};
    auto p0 = [](int a) { return a == 0 ? 1.0 : (a == 1 ? 0.0 : -1.0); };   // p_a at c = 0
    std::vector<double> N(Q), t0(Q), G(Q * Q), A(Q * Q, 0.0), Lm(Q * Q, 0.0), Y(Q * Q, 0.0), tmp(Q * Q, 0.0);
    for (int k = 0; k < Q; ++k) {
        N[k] = n1[k / 9] * n1[(k / 3) % 3] * n1[k % 3];
        t0[k] = p0(k / 9) * p0((k / 3) % 3) * p0(k % 3);
    }
    const double S = rho0 * kT / cs2, d = 3.0 * cs2 - 1.0;
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b)
            G[a * Q + b] = S * ((a == b ? 3.0 * cs2 * N[a] : 0.0) + (1.0 - 3.0 * cs2) * t0[a] * t0[b]);
    auto conserved = [](int k) { return k == 0 || k == 1 || k == 3 || k == 9; };
    for (int k = 0; k < Q; ++k) A[k * Q + k] = conserved(k) ? 0.0 : 1.0;
    for (int k : {2, 6, 18, 26}) A[k * Q + 0] = -d;          // p_2a and the sixth order follow +d rho
    for (int k : {8, 20, 24}) A[k * Q + 0] = d;              // p_2a p_2b follow -d rho
    for (int k = 0; k < Q; ++k)
        if (!conserved(k)) Lm[k * Q + k] = lg;
    for (int k : {4, 10, 12}) Lm[k * Q + k] = ls;
    for (int a : {2, 6, 18})
        for (int b : {2, 6, 18}) Lm[a * Q + b] = (lb - ls) / 3.0 + (a == b ? ls : 0.0);
    for (int a = 0; a < Q; ++a)           // tmp = A G
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;
            for (int c = 0; c < Q; ++c) s += A[a * Q + c] * G[c * Q + b];
            tmp[a * Q + b] = s;
        }
    for (int a = 0; a < Q; ++a)           // Y = A G A^T
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;
            for (int c = 0; c < Q; ++c) s += tmp[a * Q + c] * A[b * Q + c];
            Y[a * Q + b] = s;
        }
    std::vector<double> LY(Q * Q, 0.0);   // Lambda Y
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;
            for (int c = 0; c < Q; ++c) s += Lm[a * Q + c] * Y[c * Q + b];
            LY[a * Q + b] = s;
        }
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) {
            double s = 0.0;               // (Lambda Y Lambda^T)_ab
            for (int c = 0; c < Q; ++c) s += LY[a * Q + c] * Lm[b * Q + c];
            X[a * Q + b] = -(LY[b * Q + a] + LY[a * Q + b] + s);
        }
}

// lower-triangular Cholesky of the block idx[] of X (row-major, leading dimension Q); pivots
// that are zero up to 1e-12 of the block's scale are clamped; false for a negative pivot
static bool cholesky_block(const double* X, int Q, const std::vector<int>& idx, std::vector<double>& L) {
    const int n = (int)idx.size();
    L.assign((size_t)n * n, 0.0);
    double scale = 1e-300;
    for (int k : idx) scale = std::max(scale, std::fabs(X[k * Q + k]));
    for (int j = 0; j < n; ++j) {
        double s = X[idx[j] * Q + idx[j]];
        for (int q = 0; q < j; ++q) s -= L[j * n + q] * L[j * n + q];
        if (s <= 1e-12 * scale) {
            if (s < -1e-9 * scale) return false;
            continue;
        }
        L[j * n + j] = std::sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = X[idx[i] * Q + idx[j]];
            for (int q = 0; q < j; ++q) t -= L[i * n + q] * L[j * n + q];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    return true;
}

// ---- populations in and out; sums ---------------------------------------------------------

// node q of an nx x ny x nz box shifted by (sx, sy, sz) with periodic wrap (|s| <= 1)
__device__ __forceinline__ long long shifted3(long long q, int nx, int ny, int nz, int sx, int sy, int sz) {
    const long long nxy = (long long)nx * ny;
    int z = (int)(q / nxy);
    const long long r = q - (long long)z * nxy;
    int y = (int)(r / nx), x = (int)(r - (long long)y * nx);
    x += sx; y += sy; z += sz;
    x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
    return (long long)z * nxy + (long long)y * nx + x;
}

// The device holds post-collision deviations (the kernel pulls f_i(r) = f*_i(r - c_i)), so
// the pre-collision f_i(r) of the ABI is stored at r - c_i: dst(q) = f_i(q + c_i) - fbar_i.
template <typename R>
__global__ void set_plane3_kernel(const double* __restrict__ src, R* __restrict__ dst, int nx, int ny, int nz,
                                  int cx, int cy, int cz, double fbar) {
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        dst[q] = (R)(src[shifted3(q, nx, ny, nz, cx, cy, cz)] - fbar);
}

// f_i(r) = stored(r - c_i) + fbar_i
template <typename R>
__global__ void get_plane3_kernel(const R* __restrict__ src, double* __restrict__ dst, int nx, int ny, int nz,
                                  int cx, int cy, int cz, double fbar) {
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        dst[q] = (double)src[shifted3(q, nx, ny, nz, -cx, -cy, -cz)] + fbar;
}

// per-block FP64 partial sums of the density and momentum deviations
template <typename LAT, typename R>
__global__ void sums3_kernel(const R* __restrict__ p, long long n, double* __restrict__ partial) {
    double s[4] = {0, 0, 0, 0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < LAT::Q; ++i) {
            const double f = (double)p[i * n + k];
            s[0] += f;
            s[1] += LAT::c(i, 0) * f;
            s[2] += LAT::c(i, 1) * f;
            s[3] += LAT::c(i, 2) * f;
        }
    }
    __shared__ double red[4][256];
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) partial[blockIdx.x * 4 + q] = red[q][0];
}

constexpr int SUM3_BLOCKS = 256;

}  // namespace lbf3

using namespace lbf3;

struct lb3_ctx {
    int nx = 0, ny = 0, nz = 0, lattice = 19, precision = 0, device = 0, es = 4;
    long long n = 0;
    uint64_t seed = 0;
    double rho0 = 1.0, cs2 = 1.0 / 3.0;
    double fbar[QMAX] = {};
    char* ws = nullptr;
    void* pop[2] = {nullptr, nullptr};
    double* stage = nullptr;        // one FP64 plane
    double* partial = nullptr;      // SUM3_BLOCKS x 4
    int cur = 0;
    bool have_params = false;
    int noise_mode = LB_NOISE_OFF;
    double kT = 0, kappa = 0;
    Step3Args<float> af{};
    Step3Args<double> ad{};
    dim3 grid;
    bool plain = false;             // LBFLUCT3_KERNEL=plain: the plain D3Q19 kernel
    int slots = 3;                  // raw slots of the staged kernel: 3 for D3Q19, 2 for D3Q27
                                    // (the measured faster; LBFLUCT3_SLOTS=2 or 3 overrides)
    cudaStream_t stream = nullptr;
    long long t = 0;
    std::string err;
    int timing = 0;
    long long timing_seq = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t ev_used = 0;
    double ms_acc = 0.0;
    long long launches_acc = 0;
    long long kernels = 0;
};

namespace {
thread_local std::string g3_error;

int fail3(lb3_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg; else g3_error = msg;
    return code;
}

int cuda_fail3(lb3_ctx* c, cudaError_t e, const char* where) {
    return fail3(c, LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool sizes_ok(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return false;
    return (long double)nx * ny * nz < 4294967296.0L;
}

int es_of(int precision) { return precision == LB_FP32 ? 4 : (precision == LB_FP64 ? 8 : 0); }
bool lattice_ok(int lattice) { return lattice == LB_D3Q19 || lattice == LB_D3Q27; }

struct Layout3 {
    size_t pop[2], stage, partial, total;
};

Layout3 layout3(long long n, int q, int es) {
    Layout3 L{};
    size_t off = 0;
    for (int k = 0; k < 2; ++k) {
        L.pop[k] = off;
        off = align256(off + (size_t)q * n * es);
    }
    L.stage = off;
    off = align256(off + (size_t)n * sizeof(double));
    L.partial = off;
    off = align256(off + (size_t)SUM3_BLOCKS * 4 * sizeof(double));
    L.total = off;
    return L;
}

int record_timing3(lb3_ctx* c, cudaEvent_t* start, cudaEvent_t* stop) {
    if (c->ev_used == c->ev.size()) {
        if (c->ev.size() >= 1024) {
            cudaError_t e = cudaEventSynchronize(c->ev.back().second);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventSynchronize");
            for (auto& p : c->ev) {
                float ms = 0.f;
                e = cudaEventElapsedTime(&ms, p.first, p.second);
                if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventElapsedTime");
                c->ms_acc += ms;
            }
            c->ev_used = 0;
        } else {
            cudaEvent_t a, b;
            cudaError_t e = cudaEventCreate(&a);
            if (e == cudaSuccess) e = cudaEventCreate(&b);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventCreate");
            c->ev.push_back({a, b});
        }
    }
    *start = c->ev[c->ev_used].first;
    *stop = c->ev[c->ev_used].second;
    c->ev_used++;
    return LB_OK;
}

// the z run of a CTA: enough CTAs for eight per SM, each at least one plane
void choose_grid(lb3_ctx* c) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int tx = c->lattice == 19 ? Lat19::TX : Lat27::TX, ty = c->lattice == 19 ? Lat19::TY : Lat27::TY;
    const long long bxy = (long long)((c->nx + tx - 1) / tx) * ((c->ny + ty - 1) / ty);
    const long long want = 8LL * sms;
    long long chunks = std::max(1LL, std::min((long long)c->nz, (want + bxy - 1) / bxy));
    const int zc = (int)((c->nz + chunks - 1) / chunks);
    chunks = (c->nz + zc - 1) / zc;
    c->grid = dim3((c->nx + tx - 1) / tx, (c->ny + ty - 1) / ty, (unsigned)chunks);
    c->af.zc = c->ad.zc = zc;
}

// Xi(0) of the lattice, row-major Q x Q
void xi_zero(int lattice, double rho0, double cs2, double kT, double tau_s, double tau_b, double tau_g, double* X) {
    if (lattice == 19) xi_zero19(rho0, cs2, kT, -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_g, X);
    else xi_zero27(rho0, cs2, kT, -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_g, X);
}

// noise factors of the kernel: sc = sqrt of the diagonal for the uncoupled modes, Lc the
// coupled block's Cholesky factor; false if Xi(0) is not positive semidefinite
bool noise_factors(int lattice, const double* X, double sc[QMAX], double Lc[28]) {
    const int Q = lattice;
    for (int k = 0; k < QMAX; ++k) sc[k] = 0.0;
    for (int k = 0; k < 28; ++k) Lc[k] = 0.0;
    const std::vector<int> coupled = lattice == 19 ? std::vector<int>{4, 16}
                                                   : std::vector<int>(COUPLED27, COUPLED27 + 7);
    std::vector<double> L;
    if (!cholesky_block(X, Q, coupled, L)) return false;
    const int n = (int)coupled.size();
    if (lattice == 19) {
        Lc[0] = L[0];
        Lc[1] = L[1 * n + 0];
        Lc[2] = L[1 * n + 1];
    } else {
        for (int r = 0; r < n; ++r)
            for (int q = 0; q <= r; ++q) Lc[r * (r + 1) / 2 + q] = L[r * n + q];
    }
    double scale = 1e-300;
    for (int k = 0; k < Q; ++k) scale = std::max(scale, std::fabs(X[k * Q + k]));
    for (int k = 0; k < Q; ++k) {
        if (std::find(coupled.begin(), coupled.end(), k) != coupled.end()) continue;
        const double v = X[k * Q + k];
        if (v < -1e-9 * scale) return false;
        sc[k] = std::sqrt(std::max(v, 0.0));
    }
    return true;
}

template <typename R>
void fill_args(lb3_ctx* c, Step3Args<R>* a, double tau_s, double tau_b, double tau_g, const double sc[QMAX],
               const double Lc[28], const double Lrs[9]) {
    a->nx = c->nx; a->ny = c->ny; a->nz = c->nz; a->P = c->n;
    a->co.rho0 = (R)c->rho0;
    a->co.d = (R)(3.0 * c->cs2 - 1.0);
    a->co.kappa = (R)c->kappa;
    a->co.lb = (R)(-1.0 / tau_b);
    a->co.ls = (R)(-1.0 / tau_s);
    a->co.lg = (R)(-1.0 / tau_g);
    for (int q = 0; q < QMAX; ++q) a->sc[q] = (R)sc[q];
    for (int q = 0; q < 28; ++q) a->Lc[q] = (R)Lc[q];
    for (int q = 0; q < 9; ++q) a->Lrs[q] = (R)Lrs[q];
    a->rk = lbf::make_round_keys(c->seed);
}

template <typename R>
cudaError_t launch_any(lb3_ctx* c, const Step3Args<R>& a, int kmode) {
    if (c->lattice == 19) {
        if (kmode == 3) return launch3<Lat19, R, 3>(a, c->grid, false, c->slots, c->stream);
        return kmode ? launch3<Lat19, R, 1>(a, c->grid, c->plain, c->slots, c->stream)
                     : launch3<Lat19, R, 0>(a, c->grid, c->plain, c->slots, c->stream);
    }
    return kmode ? launch3<Lat27, R, 1>(a, c->grid, false, c->slots, c->stream)
                 : launch3<Lat27, R, 0>(a, c->grid, false, c->slots, c->stream);
}

}  // namespace

extern "C" {

size_t lb3_workspace_bytes(int nx, int ny, int nz, int lattice, int precision) {
    const int es = es_of(precision);
    if (!es || !lattice_ok(lattice) || !sizes_ok(nx, ny, nz)) return 0;
    return layout3((long long)nx * ny * nz, lattice, es).total;
}

int lb3_create(int nx, int ny, int nz, int lattice, int precision, uint64_t seed, double rho0, double cs2,
               lb3_ctx** out) {
    if (!out) return fail3(nullptr, LB_EINVAL, "out is NULL");
    *out = nullptr;
    const int es = es_of(precision);
    if (!lattice_ok(lattice)) return fail3(nullptr, LB_EINVAL, "lattice must be LB_D3Q19 or LB_D3Q27");
    if (!es) return fail3(nullptr, LB_EINVAL, "precision must be LB_FP32 or LB_FP64");
    if (!sizes_ok(nx, ny, nz)) return fail3(nullptr, LB_EINVAL, "sizes must be >= 1 with nx*ny*nz < 2^32");
    if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail3(nullptr, LB_EINVAL, "rho0 must be positive");
    if (!(cs2 > 0.0) || !std::isfinite(cs2)) return fail3(nullptr, LB_EINVAL, "cs2 must be positive");
    lb3_ctx* c = new lb3_ctx();
    c->nx = nx; c->ny = ny; c->nz = nz; c->n = (long long)nx * ny * nz; c->lattice = lattice;
    c->precision = precision; c->es = es; c->seed = seed; c->rho0 = rho0; c->cs2 = cs2;
    cudaGetDevice(&c->device);
    const Layout3 L = layout3(c->n, lattice, es);
    cudaError_t e = cudaMalloc((void**)&c->ws, L.total);
    if (e != cudaSuccess) {
        delete c;
        return fail3(nullptr, LB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->pop[0] = c->ws + L.pop[0];
    c->pop[1] = c->ws + L.pop[1];
    c->stage = (double*)(c->ws + L.stage);
    c->partial = (double*)(c->ws + L.partial);
    rest_pops(lattice, rho0, cs2, c->fbar);
    e = cudaMemset(c->pop[0], 0, (size_t)lattice * c->n * es);
    if (e == cudaSuccess) e = cudaMemset(c->pop[1], 0, (size_t)lattice * c->n * es);
    if (e != cudaSuccess) {
        cudaFree(c->ws);
        delete c;
        return fail3(nullptr, LB_ECUDA, std::string("lb3_create: ") + cudaGetErrorString(e));
    }
    {
        const char* v = std::getenv("LBFLUCT3_KERNEL");
        c->plain = v && std::strcmp(v, "plain") == 0 && lattice == 19;
        const char* sv = std::getenv("LBFLUCT3_SLOTS");
        c->slots = sv ? (std::atoi(sv) == 2 ? 2 : 3) : (lattice == 27 ? 2 : 3);
    }
    choose_grid(c);
    *out = c;
    return LB_OK;
}

int lb3_destroy(lb3_ctx* c) {
    if (!c) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (auto& p : c->ev) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    cudaFree(c->ws);
    delete c;
    return LB_OK;
}

int lb3_set_stream(lb3_ctx* c, void* stream) {
    if (!c) return LB_EINVAL;
    c->stream = (cudaStream_t)stream;
    return LB_OK;
}

int lb3_noise_matrix(int lattice, double rho0, double cs2, double kT, double tau_s, double tau_b, double tau_ghost,
                     double* xi) {
    if (!xi || !lattice_ok(lattice) || !(rho0 > 0) || !(cs2 > 0) || kT < 0 || !(tau_s > 0.5) || !(tau_b > 0.5) ||
        !(tau_ghost > 0.5))
        return LB_EINVAL;
    xi_zero(lattice, rho0, cs2, kT, tau_s, tau_b, tau_ghost, xi);
    return LB_OK;
}

int lb3_set_params(lb3_ctx* c, double kT, double kappa, double tau_s, double tau_b, double tau_ghost, int mode) {
    if (!c) return LB_EINVAL;
    if (!(tau_s > 0.5) || !(tau_b > 0.5) || !(tau_ghost > 0.5) || !std::isfinite(tau_s) || !std::isfinite(tau_b) ||
        !std::isfinite(tau_ghost))
        return fail3(c, LB_EINVAL, "relaxation times must exceed 1/2");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return fail3(c, LB_EINVAL, "kT must be >= 0");
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) return fail3(c, LB_EINVAL, "kappa must be >= 0");
    if (mode != LB_NOISE_OFF && mode != LB_NOISE_LW && !(mode == LB_NOISE_FULL_RS && c->lattice == 19))
        return fail3(c, LB_EINVAL, "the 3-D lattices take LB_NOISE_OFF or LB_NOISE_LW (D3Q19 also LB_NOISE_FULL_RS)");
    std::vector<double> X((size_t)c->lattice * c->lattice);
    xi_zero(c->lattice, c->rho0, c->cs2, kT, tau_s, tau_b, tau_ghost, X.data());
    double sc[QMAX] = {}, Lc[28] = {}, Lrs[9] = {};
    if (mode != LB_NOISE_OFF && kT > 0 && !noise_factors(c->lattice, X.data(), sc, Lc))
        return fail3(c, LB_ENOTPSD, "Xi(0) is not positive semidefinite");
    if (mode == LB_NOISE_FULL_RS && kT > 0) {
        // Xi(k) is Xi(0) at c_s^2(k) = cs2 + rho0 kappa s(k); the factors of its (4,16) block at
        // the corner values s = 0, 4, 16/3 (positive semidefinite there means at every k)
        const double svals[3] = {0.0, 4.0, 16.0 / 3.0};
        for (int q = 0; q < 3; ++q) {
            std::vector<double> Xs((size_t)Q3 * Q3);
            xi_zero19(c->rho0, c->cs2 + c->rho0 * kappa * svals[q], kT, -1.0 / tau_b, -1.0 / tau_s,
                      -1.0 / tau_ghost, Xs.data());
            std::vector<double> L2;
            if (!cholesky_block(Xs.data(), Q3, {4, 16}, L2))
                return fail3(c, LB_ENOTPSD, "Xi(k) is not positive semidefinite on the lattice");
            Lrs[3 * q] = L2[0];
            Lrs[3 * q + 1] = L2[2];
            Lrs[3 * q + 2] = L2[3];
        }
    }
    c->kT = kT;
    c->kappa = kappa;
    c->noise_mode = mode;
    fill_args(c, &c->af, tau_s, tau_b, tau_ghost, sc, Lc, Lrs);
    fill_args(c, &c->ad, tau_s, tau_b, tau_ghost, sc, Lc, Lrs);
    c->have_params = true;
    return LB_OK;
}

int lb3_step(lb3_ctx* c, int64_t nsteps) {
    if (!c) return LB_EINVAL;
    if (nsteps < 0) return fail3(c, LB_EINVAL, "nsteps must be >= 0");
    if (!c->have_params) return fail3(c, LB_ESTATE, "lb3_set_params must be called before lb3_step");
    lbf::DeviceGuard dg(c->device);
    const int kmode = c->kT > 0.0 ? (c->noise_mode == LB_NOISE_LW ? 1 : (c->noise_mode == LB_NOISE_FULL_RS ? 3 : 0)) : 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        const uint32_t tlo = (uint32_t)((uint64_t)c->t & 0xffffffffu), thi = (uint32_t)((uint64_t)c->t >> 32);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        const bool tm = c->timing > 0 && (c->timing_seq++ % c->timing) == 0;
        if (tm) {
            int r = record_timing3(c, &e0, &e1);
            if (r != LB_OK) return r;
            cudaError_t e = cudaEventRecord(e0, c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventRecord");
        }
        cudaError_t e;
        if (c->precision == LB_FP64) {
            Step3Args<double> a = c->ad;
            a.src = (const double*)c->pop[c->cur];
            a.dst = (double*)c->pop[c->cur ^ 1];
            a.t_lo = tlo; a.t_hi = thi;
            e = launch_any(c, a, kmode);
        } else {
            Step3Args<float> a = c->af;
            a.src = (const float*)c->pop[c->cur];
            a.dst = (float*)c->pop[c->cur ^ 1];
            a.t_lo = tlo; a.t_hi = thi;
            e = launch_any(c, a, kmode);
        }
        if (e != cudaSuccess) return cuda_fail3(c, e, "3-D step kernel launch");
        c->kernels += 1;
        if (tm) {
            e = cudaEventRecord(e1, c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventRecord");
            c->launches_acc++;
        }
        c->cur ^= 1;
        c->t++;
    }
    return LB_OK;
}

int lb3_get_time(lb3_ctx* c, int64_t* t) {
    if (!c || !t) return LB_EINVAL;
    *t = c->t;
    return LB_OK;
}

static unsigned plane_blocks(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 4096); }

int lb3_set_populations(lb3_ctx* c, const double* f, int loc, int64_t t) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE) || t < 0) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (int i = 0; i < c->lattice; ++i) {
        const double* src = f + (long long)i * c->n;
        if (loc == LB_HOST) {
            cudaError_t e = cudaMemcpyAsync(c->stage, src, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "H2D");
            src = c->stage;
        }
        const int cx = c_of(c->lattice, i, 0), cy = c_of(c->lattice, i, 1), cz = c_of(c->lattice, i, 2);
        if (c->precision == LB_FP64)
            set_plane3_kernel<double><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                src, (double*)c->pop[c->cur] + (long long)i * c->n, c->nx, c->ny, c->nz, cx, cy, cz, c->fbar[i]);
        else
            set_plane3_kernel<float><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                src, (float*)c->pop[c->cur] + (long long)i * c->n, c->nx, c->ny, c->nz, cx, cy, cz, c->fbar[i]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail3(c, e, "set populations");
        c->kernels += 1;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    c->t = t;
    return LB_OK;
}

int lb3_get_populations(lb3_ctx* c, double* f, int loc) {
    if (!c || !f || (loc != LB_HOST && loc != LB_DEVICE)) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    for (int i = 0; i < c->lattice; ++i) {
        double* dst = loc == LB_HOST ? c->stage : f + (long long)i * c->n;
        const int cx = c_of(c->lattice, i, 0), cy = c_of(c->lattice, i, 1), cz = c_of(c->lattice, i, 2);
        if (c->precision == LB_FP64)
            get_plane3_kernel<double><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                (const double*)c->pop[c->cur] + (long long)i * c->n, dst, c->nx, c->ny, c->nz, cx, cy, cz, c->fbar[i]);
        else
            get_plane3_kernel<float><<<plane_blocks(c->n), 256, 0, c->stream>>>(
                (const float*)c->pop[c->cur] + (long long)i * c->n, dst, c->nx, c->ny, c->nz, cx, cy, cz, c->fbar[i]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail3(c, e, "get populations");
        c->kernels += 1;
        if (loc == LB_HOST) {
            e = cudaMemcpyAsync(f + (long long)i * c->n, c->stage, sizeof(double) * c->n, cudaMemcpyDeviceToHost,
                                c->stream);
            if (e != cudaSuccess) return cuda_fail3(c, e, "D2H");
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    return LB_OK;
}

int lb3_sums(lb3_ctx* c, double sums[4]) {
    if (!c || !sums) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    const bool d = c->precision == LB_FP64;
    if (c->lattice == 19) {
        if (d)
            sums3_kernel<Lat19, double><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const double*)c->pop[c->cur], c->n,
                                                                           c->partial);
        else
            sums3_kernel<Lat19, float><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const float*)c->pop[c->cur], c->n,
                                                                          c->partial);
    } else {
        if (d)
            sums3_kernel<Lat27, double><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const double*)c->pop[c->cur], c->n,
                                                                           c->partial);
        else
            sums3_kernel<Lat27, float><<<SUM3_BLOCKS, 256, 0, c->stream>>>((const float*)c->pop[c->cur], c->n,
                                                                          c->partial);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail3(c, e, "sums kernel");
    c->kernels += 1;
    std::vector<double> h((size_t)SUM3_BLOCKS * 4);
    e = cudaMemcpyAsync(h.data(), c->partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "sums D2H");
    double s[4] = {0, 0, 0, 0};
    for (int b = 0; b < SUM3_BLOCKS; ++b)
        for (int q = 0; q < 4; ++q) s[q] += h[(size_t)b * 4 + q];
    sums[0] = c->rho0 * (double)c->n + s[0];
    sums[1] = s[1];
    sums[2] = s[2];
    sums[3] = s[3];
    return LB_OK;
}

int lb3_set_kernel_timing(lb3_ctx* c, int every) {
    if (!c) return LB_EINVAL;
    if (every < 0) return fail3(c, LB_EINVAL, "timing stride must be >= 0");
    c->timing = every;
    c->timing_seq = 0;
    c->ev_used = 0;
    c->ms_acc = 0.0;
    c->launches_acc = 0;
    return LB_OK;
}

int lb3_kernel_time(lb3_ctx* c, double* ms, int64_t* launches) {
    if (!c) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    double total = c->ms_acc;
    if (c->ev_used > 0) {
        cudaError_t e = cudaEventSynchronize(c->ev[c->ev_used - 1].second);
        if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventSynchronize");
        for (size_t k = 0; k < c->ev_used; ++k) {
            float v = 0.f;
            e = cudaEventElapsedTime(&v, c->ev[k].first, c->ev[k].second);
            if (e != cudaSuccess) return cuda_fail3(c, e, "cudaEventElapsedTime");
            total += v;
        }
    }
    if (ms) *ms = total;
    if (launches) *launches = c->launches_acc;
    return LB_OK;
}

int lb3_launch_count(lb3_ctx* c, int64_t* launches) {
    if (!c || !launches) return LB_EINVAL;
    *launches = c->kernels;
    return LB_OK;
}

int lb3_synchronize(lb3_ctx* c) {
    if (!c) return LB_EINVAL;
    lbf::DeviceGuard dg(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "cudaStreamSynchronize");
    return LB_OK;
}

const char* lb3_last_error(lb3_ctx* c) { return c ? c->err.c_str() : g3_error.c_str(); }

}  // extern "C"
