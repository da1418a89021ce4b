// lb3d_kernel.cuh -- the fused fluctuating step kernels of the D3Q19 and D3Q27 lattices for
// sm_103a (one launch per time step: collision of lb3_collide.cuh or lb27_collide.cuh, then
// streaming in pull form, f_i(r, t) = f*_i(r - c_i, t - 1)).
//
// Storage.  Each population plane of the nx x ny x nz lattice is kept with periodic ghost
// copies: gx ghost columns on either side of a row (the host takes 32 bytes of elements, so
// that the interior of every row starts on a 32-byte sector) and GY3 = 2 ghost rows below and
// above every z plane.  Population i lives in plane sigma(i) of its buffer; element
// (plane s, x, y, z), -gx <= x < nx + gx, -GY3 <= y < ny + GY3, lives at
//   s P + z PL + (y + GY3) pitch + (x + gx),
// pitch = nx + 2 gx rounded up to a multiple of gx, PL = (ny + 2 GY3) pitch, P = nz PL.  The
// step writes every node's ghost copies with the node (columns GW = 32 bytes of elements
// wide, so that the copies of an edge warp fill whole sectors), so each read of the next
// step, f*_i(r - c_i) for r on a tile's one-node ring, is a wrap-free address in x and y; z
// wraps by plane.
//
// The staged kernel.  A CTA owns a TX x TY tile of the (x, y) plane and marches over a run
// of z planes.  The pulled populations of each plane, for the tile and its one-node ring,
// are staged in shared memory, either by TMA (one 4-D box per population, issued by one
// thread and completed on an mbarrier per slot) or by asynchronous 4- or 8-byte copies
// (cp.async) issued by every thread.  Three rotating slots hold the plane being collided,
// the plane whose densities are summed, and the plane in flight, so the loads of plane z+2
// overlap the collision of plane z; with two slots a plane's own populations move to
// registers when its densities are summed, which frees its slot for the plane after next.
// The densities of planes z-1, z, z+1 sit in three more rotating slots; the collision reads
// its node's populations and its 3x3x3 density neighbourhood from shared memory.  Every
// population is read once from DRAM (the ring's re-reads hit L2) and written once, plus the
// ghost copies.
//
// A plain D3Q19 kernel (density summed from direct loads, the collision pulling again) is
// kept as a cross-check.
#pragma once

#include <cuda.h>

#include <atomic>

#include "lb27_collide.cuh"
#include "lb3_collide.cuh"
#include "lb_internal.cuh"
#include "lb_tma.cuh"

namespace lbf3 {

constexpr int QMAX = 27;

// velocity components in {-1, 0, 1} packed two bits each: c = ((P >> 2i) & 3) - 1
constexpr unsigned long long pack3(const int (&v)[19]) {
    unsigned long long p = 0;
    for (int i = 0; i < 19; ++i) p |= (unsigned long long)(v[i] + 1) << (2 * i);
    return p;
}

// Each lattice stores population i in plane sigma(i) of its buffer; the TMA staging loads the
// populations of one box together, GM consecutive planes that share c_y and c_z.
// D3Q19: the velocity order of lb3_collide.cuh; noise tags 4, 5; one population per box
struct Lat19 {
    static constexpr int Q = 19, TX = 32, GM = 1;
    static constexpr uint32_t TAG0 = 4;
    static constexpr int CXv[19] = {0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
    static constexpr int CYv[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 0, 0, 0, 0};
    static constexpr int CZv[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1};
    static constexpr unsigned long long PX = pack3(CXv), PY = pack3(CYv), PZ = pack3(CZv);
    __host__ __device__ static constexpr int c(int i, int k) {
        return (int)(((k == 0 ? PX : (k == 1 ? PY : PZ)) >> (2 * i)) & 3ULL) - 1;
    }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
    __host__ __device__ static constexpr int sigma(int i) { return i; }
    __host__ __device__ static constexpr int box(int i) { return i; }
    __host__ __device__ static constexpr int member(int) { return 0; }
};

// D3Q27: i = 9 ix + 3 iy + iz, components (0, 1, -1); noise tags 6, 7, 8; stored in plane
// sigma(i) = 3 (3 iy + iz) + ix, so that the three populations of one (c_y, c_z) are
// consecutive planes and one box (i mod 9 = 3 iy + iz) carries all three
struct Lat27 {
    static constexpr int Q = 27, TX = 32, GM = 3;
    static constexpr uint32_t TAG0 = 6;
    __host__ __device__ static constexpr int v(int a) { return a == 0 ? 0 : (a == 1 ? 1 : -1); }
    __host__ __device__ static constexpr int c(int i, int k) {
        return v(k == 0 ? i / 9 : (k == 1 ? (i / 3) % 3 : i % 3));
    }
    __host__ __device__ static constexpr double w1(int a) { return a == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double w(int i) { return w1(i / 9) * w1((i / 3) % 3) * w1(i % 3); }
    __host__ __device__ static constexpr int sigma(int i) { return 3 * (i % 9) + i / 9; }
    __host__ __device__ static constexpr int box(int i) { return i % 9; }
    __host__ __device__ static constexpr int member(int i) { return i / 9; }
};

// The D3Q27 modes whose noise is coupled (the Cholesky factor's dense 7 x 7 block, in mode
// order): p_2z, p_2y, p_2y p_2z, p_2x, p_2x p_2z, p_2x p_2y, p_2x p_2y p_2z.
constexpr int COUPLED27[7] = {2, 6, 8, 18, 20, 24, 26};
__host__ __device__ constexpr int coupled27(int r) {
    return r == 0 ? 2 : (r == 1 ? 6 : (r == 2 ? 8 : (r == 3 ? 18 : (r == 4 ? 20 : (r == 5 ? 24 : 26)))));
}

// ghost columns written per side (32 bytes of elements: one sector) and ghost rows per side
template <typename R>
__host__ __device__ constexpr int gw3() { return 32 / (int)sizeof(R); }
constexpr int GY3 = 2;

template <typename R>
struct Step3Args {
    const R* __restrict__ src;    // post-collision deviations at t-1 (padded storage above)
    R* __restrict__ dst;
    int nx, ny, nz, zc;           // zc: planes per CTA
    int pitch;                    // elements per stored row
    int gx;                       // stored column of x = 0
    long long PL;                 // elements per stored z plane
    long long P;                  // elements per population (nz PL)
    int* err;                     // device error word: 1 = a CTA gave up waiting for its TMA loads
    Coef3<R> co;
    R sc[QMAX];                   // sqrt(Xi_kk) of the modes with a diagonal factor (local noise:
                                  // per unit density)
    R Lc[28];                     // the coupled block's Cholesky factor: D3Q19 (L44, L16_4, L16_16);
                                  // D3Q27 the 7 x 7 lower triangle, row-major.  Local noise: A of
                                  // its Xi(0) = rho (A + B c_s^2), same layout
    R Lb[28];                     // local noise: B of the coupled block
    R cq[4];                      // local noise: c_s^2(rho0 + dr) = cq0 + dr (cq1 + dr (cq2 + dr cq3))
    R Lrs[12];                    // correlated noise, per corner class (L11, L21, L22): D3Q19 the
                                  // Cholesky factors of the (4,16) block of Xi at s = 0, 4, 16/3;
                                  // D3Q27 (sqrt(s), 0, sqrt(S - s)) at s = 0, 4, 16/3, 52/9 = S
    R Prs[7], Qrs[7];             // D3Q27 correlated noise: the coupled modes' directions p, q of
                                  // the box-filtered fields (Lc then factors the white part)
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

// D3Q19 noise at the local density (MODE 4, Sec. IV and Sec. V B): the draws of normals19;
// Xi(0) of a homogeneous system at this node's density rho0 + dr and sound speed
// c_s^2(rho0 + dr) is rho (A + B c_s^2) entrywise (A, B from the host); the (4,16) block is
// factored here by Cholesky with a negative pivot clamped to zero, the other modes scale with
// sqrt(rho)
template <typename R>
__device__ __forceinline__ void normals19_local(const Step3Args<R>& a, uint32_t node, R dr, R xi[Q3]) {
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
    const R rho = a.co.rho0 + dr;
    const R c = a.cq[0] + dr * (a.cq[1] + dr * (a.cq[2] + dr * a.cq[3]));
    const R sr = lbf::sqrt_fast(fmax(rho, R(0)));
#pragma unroll
    for (int q = 5; q < Q3; ++q) xi[q] *= sr * a.sc[q];
    const R y44 = rho * (a.Lc[0] + a.Lb[0] * c);
    const R y416 = rho * (a.Lc[1] + a.Lb[1] * c);
    const R y1616 = rho * (a.Lc[2] + a.Lb[2] * c);
    const R L44 = lbf::sqrt_fast(fmax(y44, R(0)));
    const R L164 = L44 > R(0) ? y416 * lbf::recip(L44) : R(0);
    const R L1616 = lbf::sqrt_fast(fmax(y1616 - L164 * L164, R(0)));
    xi[4] = L44 * n4;
    xi[16] = L164 * n4 + L1616 * n16;
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

// D3Q27 noise at the local density (MODE 4): the draws of normals27; the uncoupled modes scale
// with sqrt(rho), the seven coupled modes take the Cholesky factor, formed here, of the block
// rho (A + B c_s^2) (a negative pivot clamped to zero leaves its column zero)
template <typename R>
__device__ __forceinline__ void normals27_local(const Step3Args<R>& a, uint32_t node, R dr, R xi[Q27]) {
    R nu[24];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const uint4 r = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, Lat27::TAG0 + d), a.rk);
        lbf::gauss_word(r.x, &nu[8 * d + 0], &nu[8 * d + 1]);
        lbf::gauss_word(r.y, &nu[8 * d + 2], &nu[8 * d + 3]);
        lbf::gauss_word(r.z, &nu[8 * d + 4], &nu[8 * d + 5]);
        lbf::gauss_word(r.w, &nu[8 * d + 6], &nu[8 * d + 7]);
    }
    const R rho = a.co.rho0 + dr;
    const R c = a.cq[0] + dr * (a.cq[1] + dr * (a.cq[2] + dr * a.cq[3]));
    const R sr = lbf::sqrt_fast(fmax(rho, R(0)));
#pragma unroll
    for (int k = 0; k < Q27; ++k)
        xi[k] = (k == 0 || k == 1 || k == 3 || k == 9) ? R(0) : sr * a.sc[k] * nu[nc27(k)];
    R L[28], inv[7];
#pragma unroll
    for (int r = 0; r < 7; ++r) {
#pragma unroll
        for (int q = 0; q <= r; ++q) {
            const int e = r * (r + 1) / 2 + q;
            R y = rho * (a.Lc[e] + a.Lb[e] * c);
#pragma unroll
            for (int p = 0; p < q; ++p) y -= L[r * (r + 1) / 2 + p] * L[q * (q + 1) / 2 + p];
            if (q == r) {
                L[e] = lbf::sqrt_fast(fmax(y, R(0)));
                inv[r] = L[e] > R(0) ? lbf::recip(L[e]) : R(0);
            } else {
                L[e] = y * inv[q];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 7; ++r) {
        R s = R(0);
#pragma unroll
        for (int q = 0; q <= r; ++q) s += L[r * (r + 1) / 2 + q] * nu[nc27(coupled27(q))];
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

// Writes the Q post-collision values of node (x, y) of the stored plane at offset zo, and its
// ghost copies: columns x + nx (x < GW) or x - nx (x >= nx - GW), rows y + ny (y < GY3) or
// y - ny (y >= ny - GY3), and the corner.  On lattices narrower than 2 GW or lower than
// 2 GY3 a node can feed several copies per side; those go through the general loop.  Indices
// are formed in I (32-bit when all planes fit in 2^32 elements) with modular arithmetic, so
// negative displacements are added as their two's complement.
template <typename LAT, typename R, typename I>
__device__ __forceinline__ void store_node3(const Step3Args<R>& a, I zo, int x, int y, const R (&o)[LAT::Q]) {
    constexpr int Q = LAT::Q;
    constexpr int GW = gw3<R>();
    const int nx = a.nx, ny = a.ny, pitch = a.pitch, gx = a.gx;
    const I PI = (I)a.P;
    R* __restrict__ d = a.dst;
    const I ns = zo + (I)(y + GY3) * (I)pitch + (I)(x + gx);
    if (nx >= 2 * GW && ny >= 2 * GY3) {
        const bool hx = x < GW || x >= nx - GW, hy = y < GY3 || y >= ny - GY3;
        if (!(hx | hy)) {
#pragma unroll
            for (int i = 0; i < Q; ++i) d[(I)LAT::sigma(i) * PI + ns] = o[i];
        } else {
            const I dx = hx ? (I)(long long)(x < GW ? nx : -nx) : (I)0;
            const I dy = hy ? (I)((long long)(y < GY3 ? ny : -ny) * pitch) : (I)0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const I b = (I)LAT::sigma(i) * PI + ns;
                d[b] = o[i];
                if (hx) d[b + dx] = o[i];
                if (hy) d[b + dy] = o[i];
                if (hx & hy) d[b + dx + dy] = o[i];
            }
        }
    } else {
        // every column cx = x (mod nx) in [-GW, nx + GW) and row cy = y (mod ny) in [-GY3, ny + GY3)
        const int cy0 = y - ((y + GY3) / ny) * ny, cx0 = x - ((x + GW) / nx) * nx;
        for (int cy = cy0; cy < ny + GY3; cy += ny)
            for (int cx = cx0; cx < nx + GW; cx += nx) {
                const I b = zo + (I)(cy + GY3) * (I)pitch + (I)(cx + gx);
#pragma unroll
                for (int i = 0; i < Q; ++i) d[(I)LAT::sigma(i) * PI + b] = o[i];
            }
    }
}

// correlated noise: the first of the two tags of the draws of the eight corner fields (word w
// -> the pair of corner w: D3Q19 the white 2-vector of the (4,16) block, D3Q27 the white
// values of the two scalar fields along p and q), the pair's components, and the corner
// class of a corner with pc components at pi (the table row of Lrs)
constexpr uint32_t TAG_RS0 = 10;
constexpr uint32_t TAG_RS27 = 12;
constexpr int RS_NV = 2;
template <typename LAT>
__host__ __device__ constexpr uint32_t rs_tag() { return LAT::Q == 19 ? TAG_RS0 : TAG_RS27; }
template <typename LAT>
__host__ __device__ constexpr int rs_class(int pc) { return LAT::Q == 19 ? (pc == 0 ? 0 : (pc == 2 ? 2 : 1)) : pc; }

// Shared-memory geometry of one raw slot.  Copies (TMA = false): per population the pulled
// values of the tile and its ring, RX x RY, already shifted by -c_i.  TMA: per box the GM
// populations of one (c_y, c_z), each BW x RY stored values whose origin is (x0 - XO,
// y0 - 1 - c_iy, z - c_iz), XO = 16 bytes of elements (the TMA x alignment; x0 + gx - XO is
// then a multiple of XO); the pulled value at ring position (qx, qy) is
// pop[qy][qx - 1 + XO - c_ix].  Every box starts on 128 bytes.
template <typename LAT, typename R, int TY, bool TMA>
struct Slot3 {
    static constexpr int TX = LAT::TX, RX = TX + 2, RY = TY + 2, RN = RX * RY;
    static constexpr int XO = 16 / (int)sizeof(R);
    static constexpr int BW = TMA ? TX + 2 * XO : RX;           // row width in the slot
    static constexpr int NB = LAT::Q / LAT::GM;                 // TMA boxes per plane
    static constexpr int BOX_BYTES = LAT::GM * (TX + 2 * XO) * RY * (int)sizeof(R);
    static constexpr int PB = ((BOX_BYTES + 127) / 128) * 128 / (int)sizeof(R);   // box stride
    static constexpr int SLOT = TMA ? NB * PB : LAT::Q * RN;    // elements per slot
    // first element of population i in a slot
    __host__ __device__ static constexpr int pbase(int i) {
        return TMA ? LAT::box(i) * PB + LAT::member(i) * RY * BW : i * RN;
    }
    __host__ __device__ static constexpr int col(int cx) { return TMA ? XO - 1 - cx : 0; }
};

// Shared memory of the staged kernel: [SLOTS][SLOT] raw values, the mbarriers (TMA), the
// density ring [3][RN], and with correlated noise (MODE 3) the 2x2x2-box contributions: for
// the tile plus its left column and bottom row, the in-plane half (four pairs) of the current
// plane and the upward half of the current and the previous plane.
template <typename LAT, typename R, int TY, int SLOTS, int MODE, bool TMA>
constexpr int staged_smem_bytes() {
    using S = Slot3<LAT, R, TY, TMA>;
    constexpr int HV = MODE == 3 ? 12 * RS_NV * (LAT::TX + 1) * (TY + 1) : 0;
    return (SLOTS * S::SLOT + 3 * S::RN + HV) * (int)sizeof(R) + (TMA ? 16 * ((SLOTS + 1) / 2) : 0);
}

// resident CTAs per SM the register budget is sized for: as many as the shared memory admits
// (228 KB per SM, 1 KB reserved per CTA), at most 2048 threads
template <typename LAT, typename R, int TY, int SLOTS, int MODE, bool TMA>
constexpr int staged_min_blocks() {
    constexpr int by_smem = (228 * 1024) / (staged_smem_bytes<LAT, R, TY, SLOTS, MODE, TMA>() + 1024);
    constexpr int by_threads = 2048 / (LAT::TX * TY);
    return by_smem < 1 ? 1 : (by_smem < by_threads ? by_smem : by_threads);
}

template <typename LAT, typename R, int TY, int MODE, typename I, int SLOTS, bool TMA>
__global__ void __launch_bounds__(LAT::TX * TY, staged_min_blocks<LAT, R, TY, SLOTS, MODE, TMA>())
    step3_staged_kernel(const __grid_constant__ CUtensorMap tmap, const Step3Args<R> a) {
    constexpr int Q = LAT::Q, TX = LAT::TX;
    using S = Slot3<LAT, R, TY, TMA>;
    constexpr int RX = S::RX, RN = S::RN, NT = TX * TY, SL = S::SLOT, BW = S::BW;
    extern __shared__ __align__(128) unsigned char smem3[];
    R* raw = reinterpret_cast<R*>(smem3);                                   // [SLOTS][SL]
    constexpr int RAW_BYTES = SLOTS * SL * (int)sizeof(R);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem3 + RAW_BYTES);         // TMA: one per slot
    R* rs = reinterpret_cast<R*>(smem3 + RAW_BYTES + (TMA ? 16 * ((SLOTS + 1) / 2) : 0));   // [3][RN]
    constexpr int HW = TX + 1, HN = HW * (TY + 1), NV = RS_NV;
    R* Hin = rs + 3 * RN;                                   // MODE 3: [4][NV][HN] in-plane half
    R* Hup = Hin + 4 * NV * HN;                             // MODE 3: [2][4][NV][HN] upward half
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch, GX = a.gx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, nz);
    const int tid = threadIdx.x;
    const R* __restrict__ src = a.src;
    // offsets in I: 32-bit when all Q populations fit in 2^32 elements, else 64-bit
    const I PI = (I)a.P, PLI = (I)a.PL;

    if constexpr (TMA) {
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < SLOTS; ++k) lbf::mbar_init(lbf::smem_u32(&bar[k]), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
        }
        __syncthreads();
    }

    // Copies: the ring positions a thread stages are the same on every plane; their stored
    // in-plane offsets (no wrap: the ghosts cover the ring) and validity are formed once.
    constexpr int KP = (RN + NT - 1) / NT;
    I base[KP];
    bool valid[KP];
    if constexpr (!TMA) {
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int q = tid + k * NT;
            const int ly = q / RX, lx = q - ly * RX;
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            valid[k] = q < RN && gx <= nx && gy <= ny;      // others are never read by a node
            base[k] = (I)(gy + GY3) * (I)pitch + (I)(gx + GX);
        }
    }

    uint32_t phase = 0;      // TMA: parity of each slot's next completion (bit k)
    uint32_t pending = 0;    // TMA, thread 0: slots with loads in flight (bit k)

    // issue the pulled populations of plane zz (an integer in [-1, nz]) into raw slot k
    auto issue = [&](int zz, int slot_k) {
        const int zc = wrap_hi(wrap_lo(zz, nz), nz);
        const int Zc[3] = {zc == 0 ? nz - 1 : zc - 1, zc, zc == nz - 1 ? 0 : zc + 1};   // z - cz, by 1 - cz
        R* slot = raw + slot_k * SL;
        if constexpr (TMA) {
            if (tid != 0) return;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const uint32_t b = lbf::smem_u32(&bar[slot_k]);
            lbf::mbar_expect_tx(b, (uint32_t)(S::NB * S::BOX_BYTES));
            // box j holds the populations of the same c_y, c_z as population j (its first member)
#pragma unroll
            for (int j = 0; j < S::NB; ++j)
                lbf::tma_load_4d(lbf::smem_u32(slot + j * S::PB), &tmap, x0 - S::XO + GX, y0 - 1 - LAT::c(j, 1) + GY3,
                                 Zc[1 - LAT::c(j, 2)], LAT::sigma(j), b);
            pending |= 1u << slot_k;
        } else {
            const I Zo[3] = {(I)Zc[0] * PLI, (I)Zc[1] * PLI, (I)Zc[2] * PLI};
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                if (!valid[k]) continue;
                const int q = tid + k * NT;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const I dyx = (I)(long long)(-(LAT::c(i, 1) * pitch + LAT::c(i, 0)));
                    const I off = (I)LAT::sigma(i) * PI + Zo[1 - LAT::c(i, 2)] + base[k] + dyx;
                    cp_async_elem<sizeof(R)>(slot + S::pbase(i) + q, src + off);
                }
            }
            cp_async_commit();
        }
    };
    // wait until raw slot k has landed and is visible to the whole CTA (a block-wide barrier
    // either way); false, for every thread, if any thread gave up on a TMA wait
    auto wait_slot = [&](int slot_k) -> bool {
        if constexpr (TMA) {
            const uint32_t par = (phase >> slot_k) & 1u;
            const bool ok = lbf::mbar_wait_bounded(lbf::smem_u32(&bar[slot_k]), par);
            if (__syncthreads_or(!ok)) return false;
            phase ^= 1u << slot_k;
            pending &= ~(1u << slot_k);
            return true;
        } else {
            cp_async_wait_all();
            __syncthreads();
            return true;
        }
    };
    // a CTA that gave up sets the error word and gives its loads in flight a bounded chance
    // to land in its shared memory before it exits
    auto give_up = [&]() {
        if constexpr (TMA) {
            if (tid == 0) {
                atomicExch(a.err, 1);
#pragma unroll
                for (int k = 0; k < SLOTS; ++k)
                    if ((pending >> k) & 1u) lbf::mbar_wait_bounded(lbf::smem_u32(&bar[k]), (phase >> k) & 1u);
            }
        }
    };
    // density deviations of the plane in raw slot slot_k into density slot dk; positions run
    // from the last thread down, so the positions beyond the block's width fall on other
    // threads than the extra copies of issue()
    auto density = [&](int slot_k, int dk) {
        const R* slot = raw + slot_k * SL;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int q = (NT - 1 - tid) + k * NT;
            if (q >= RN) continue;
            const int ly = q / RX, lx = q - ly * RX;
            R v = R(0);
            if (x0 + lx - 1 <= nx && y0 + ly - 1 <= ny) {
                const int b = ly * BW + lx;
                R f[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) f[i] = slot[S::pbase(i) + b + S::col(LAT::c(i, 0))];
                v = drho_of<LAT>(f);
            }
            rs[dk * RN + q] = v;
        }
    };

    const int lx = tid % TX, ly = tid / TX;
    const int x = x0 + lx, y = y0 + ly;
    const bool own = x < nx && y < ny;
    const int qc = (ly + 1) * RX + lx + 1;     // own position in the density ring
    const int qb = (ly + 1) * BW + lx + 1;     // own position in a raw slot

    // MODE 3: the eight white pairs nu_w of every position of plane zz (tile, left column,
    // bottom row), times the factor of their corner class (w = 4 ia + 2 ib + ic, sign -1 for a
    // set bit: k = pi), combined by a Walsh-Hadamard transform into h_m = (1/8) sum_w
    // (-1)^{popcount(w & m)} L_w nu_w, m = 4 dx + 2 dy + dz: the in-plane half (dz = 0) into Hin
    // when keep_in, the upward half (dz = 1) into buffer ub.  D3Q19: the (4,16) block's
    // 2-vector; D3Q27: the two scalar fields along p and q (L_w diagonal)
    auto stencil_plane = [&](int zz, bool keep_in, int ub) {
        const int zc = wrap_hi(wrap_lo(zz, nz), nz);
        for (int p = NT - 1 - tid; p < HN; p += NT) {       // extra positions on the last threads
            const int hy = p / HW - 1, hx = p - (hy + 1) * HW - 1;
            int gx = x0 + hx, gy = y0 + hy;
            if (gx >= nx || gy >= ny) continue;         // never read by a node of the lattice
            gx = wrap_lo(gx, nx);
            gy = wrap_lo(gy, ny);
            const uint32_t node = ((uint32_t)zc * (uint32_t)ny + (uint32_t)gy) * (uint32_t)nx + (uint32_t)gx;
            const uint4 r0 = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, rs_tag<LAT>()), a.rk);
            const uint4 r1 = lbf::philox4x32_10(make_uint4(node, a.t_lo, a.t_hi, rs_tag<LAT>() + 1), a.rk);
            const uint32_t wd[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            R vx[8], vy[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                R n0, n1;
                lbf::gauss_word(wd[w], &n0, &n1);
                const int cls = rs_class<LAT>((w & 1) + ((w >> 1) & 1) + ((w >> 2) & 1));
                vx[w] = a.Lrs[3 * cls] * n0;
                if constexpr (LAT::Q == 19)
                    vy[w] = a.Lrs[3 * cls + 1] * n0 + a.Lrs[3 * cls + 2] * n1;
                else
                    vy[w] = a.Lrs[3 * cls + 2] * n1;
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
                R* dst = (m & 1) ? Hup + ub * 4 * NV * HN : Hin;
                if (!(m & 1) && !keep_in) continue;
                const int j = m >> 1;
                dst[(j * NV) * HN + p] = R(0.125) * vx[m];
                dst[(j * NV + 1) * HN + p] = R(0.125) * vy[m];
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
        const uint32_t node = ((uint32_t)z * (uint32_t)ny + (uint32_t)y) * (uint32_t)nx + (uint32_t)x;
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
            if (MODE == 1 || MODE == 3) normals19(a, node, xi);
            if (MODE == 4) normals19_local(a, node, r.c, xi);
            if constexpr (MODE == 3) {
                // (xi_4, xi_16) = sum over the box: h of r - (dx, dy, 0) from this plane and of
                // r - (dx, dy, 1) from the previous one
                R s4 = R(0), s16 = R(0);
                const R* hu = Hup + hb * 4 * NV * HN;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int q = (ly - (j & 1) + 1) * HW + (lx - (j >> 1) + 1);
                    s4 += Hin[(j * NV) * HN + q] + hu[(j * NV) * HN + q];
                    s16 += Hin[(j * NV + 1) * HN + q] + hu[(j * NV + 1) * HN + q];
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
            if (MODE == 1 || MODE == 3) normals27(a, node, xi);
            if (MODE == 4) normals27_local(a, node, nb[0], xi);
            if constexpr (MODE == 3) {
                // the coupled modes: the white part (normals27 with the factor of C) plus p phi_p
                // + q phi_q, the two fields the 2x2x2-box sums of this plane's in-plane halves
                // and the previous plane's upward halves
                R sp = R(0), sq = R(0);
                const R* hu = Hup + hb * 4 * NV * HN;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int q = (ly - (j & 1) + 1) * HW + (lx - (j >> 1) + 1);
                    sp += Hin[(j * NV) * HN + q] + hu[(j * NV) * HN + q];
                    sq += Hin[(j * NV + 1) * HN + q] + hu[(j * NV + 1) * HN + q];
                }
#pragma unroll
                for (int r = 0; r < 7; ++r) xi[coupled27(r)] += a.Prs[r] * sp + a.Qrs[r] * sq;
            }
            collide27(a.co, f, nb, xi, o);
        }
        store_node3<LAT, R, I>(a, (I)z * PLI, x, y, o);
    };

    if constexpr (SLOTS == 3) {
        // planes z0-1, z0 -> slots 0, 1; plane z0+1 -> slot 2 (in flight); density slots alike
        issue(z0 - 1, 0);
        issue(z0, 1);
        if constexpr (TMA) issue(z0 + 1, 2);
        if (!wait_slot(0) || !wait_slot(1)) { give_up(); return; }
        density(0, 0);
        density(1, 1);
        if constexpr (MODE == 3) stencil_plane(z0 - 1, false, 0);
        if constexpr (!TMA) issue(z0 + 1, 2);
        for (int z = z0; z < z1; ++z) {
            const int k0 = (z - z0 + 1) % 3, km = (k0 + 2) % 3, kp = (k0 + 1) % 3;   // slots of z, z-1, z+1
            if (!wait_slot(kp)) { give_up(); return; }
            if (TMA && z + 1 < z1) issue(z + 2, km);    // plane z-1's slot is free
            density(kp, kp);
            if constexpr (MODE == 3) stencil_plane(z, true, (z - z0 + 1) & 1);
            if (!TMA && z + 1 < z1) issue(z + 2, km);
            __syncthreads();
            if (!own) continue;
            const R* sl = raw + k0 * SL;
            R f[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = sl[S::pbase(i) + qb + S::col(LAT::c(i, 0))];
            collide_plane(z, f, k0, km, kp, (z - z0) & 1);
        }
    } else {
        // two raw slots: a plane's own pulled values move to registers when its densities are
        // summed, which frees its slot for the plane after next
        R fcur[Q], fnext[Q];
        auto take = [&](int k, R (&f)[Q]) {
            const R* sl = raw + k * SL;
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = own ? sl[S::pbase(i) + qb + S::col(LAT::c(i, 0))] : R(0);
        };
        issue(z0 - 1, 0);
        issue(z0, 1);
        if (!wait_slot(0) || !wait_slot(1)) { give_up(); return; }
        density(0, 0);                 // plane z0-1 -> density slot 0
        density(1, 1);                 // plane z0 -> density slot 1
        take(1, fcur);
        if constexpr (MODE == 3) stencil_plane(z0 - 1, false, 0);
        __syncthreads();
        issue(z0 + 1, 0);              // raw slot of plane p: (p - z0 + 1) % 2
        for (int z = z0; z < z1; ++z) {
            const int k0 = (z - z0 + 1) % 3, km = (k0 + 2) % 3, kp = (k0 + 1) % 3;
            const int rp = (z - z0) & 1;             // raw slot of plane z+1
            if (!wait_slot(rp)) { give_up(); return; }
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
    if constexpr (!TMA) cp_async_wait_all();
}

// ---- the plain D3Q19 kernel (cross-check) -----------------------------------------------

// the 19 pulled deviations of the node at stored in-plane offset b: f_i = src_i(r - c_i),
// Zs[1 - cz] the stored offsets of planes z - 1, z, z + 1
template <typename R>
__device__ __forceinline__ void pull19(const R* __restrict__ s, long long P, const long long (&Zs)[3], long long b,
                                       int pitch, R f[Q3]) {
#pragma unroll
    for (int i = 0; i < Q3; ++i)
        f[i] = s[i * P + Zs[1 - Lat19::c(i, 2)] + b - (long long)Lat19::c(i, 1) * pitch - Lat19::c(i, 0)];
}

template <typename R, int MODE, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) step3_kernel(const Step3Args<R> a) {
    constexpr int RX = TX + 2, RY = TY + 2, NT = TX * TY;
    __shared__ R rs[3][RY][RX];
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch, GX = a.gx;
    const long long P = a.P, PL = a.PL;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, nz);
    const int tid = threadIdx.x;
    const R* __restrict__ src = a.src;
    auto planes = [&](int zz, long long (&Zs)[3]) {
        const int zc = wrap_hi(wrap_lo(zz, nz), nz);
        Zs[0] = (zc == 0 ? nz - 1 : zc - 1) * PL;
        Zs[1] = zc * PL;
        Zs[2] = (zc == nz - 1 ? 0 : zc + 1) * PL;
    };

    auto density = [&](int zz, int slot) {
        long long Zs[3];
        planes(zz, Zs);
        for (int q = tid; q < RX * RY; q += NT) {
            const int ly = q / RX, lx = q - ly * RX;
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            R v = R(0);
            if (gx <= nx && gy <= ny) {
                R f[Q3];
                pull19(src, P, Zs, (long long)(gy + GY3) * pitch + gx + GX, pitch, f);
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
    const long long b = (long long)(y + GY3) * pitch + x + GX;
    for (int z = z0; z < z1; ++z) {
        const int s0 = (z - z0 + 1) % 3, sm = (s0 + 2) % 3, sp = (s0 + 1) % 3;
        density(z + 1, sp);
        __syncthreads();
        if (own) {
            long long Zs[3];
            planes(z, Zs);
            R f[Q3];
            pull19(src, P, Zs, b, pitch, f);
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
            const uint32_t node = ((uint32_t)z * (uint32_t)ny + (uint32_t)y) * (uint32_t)nx + (uint32_t)x;
            if (MODE == 1) normals19(a, node, xi);
            R o[Q3];
            collide19(a.co, f, r, xi, o);
            store_node3<Lat19, R, long long>(a, z * PL, x, y, o);
        }
        __syncthreads();
    }
}

// ---- launch ---------------------------------------------------------------------------------

// The launch configuration of a context: grid, kernel noise mode (0 off, 1 Xi(0), 3 the
// correlated noise of D3Q19, 4 Xi(0) at the local density), the staged kernel's raw slots, staging (TMA or copies) and tile
// height, or the plain D3Q19 kernel.
struct Launch3 {
    dim3 grid;
    int zc;            // planes per CTA
    int kmode;
    int slots;
    bool tma;
    int ty;
    bool plain;
};

template <typename LAT, typename R, int TY, int MODE, typename I, int SLOTS, bool TMA>
static cudaError_t launch_staged(const Step3Args<R>& a, const CUtensorMap* map, dim3 grid, cudaStream_t s) {
    constexpr int smem = staged_smem_bytes<LAT, R, TY, SLOTS, MODE, TMA>();
    if constexpr (smem > 227 * 1024) {
        return cudaErrorInvalidConfiguration;      // this variant's shared memory does not fit a CTA
    } else {
        auto kern = step3_staged_kernel<LAT, R, TY, MODE, I, SLOTS, TMA>;
        // the shared-memory limit is a per-device attribute of the function: set it once per
        // device (a repeated set from a concurrent first launch is harmless)
        static std::atomic<unsigned> done{0};
        int dev = 0;
        cudaGetDevice(&dev);
        const unsigned bit = 1u << (dev & 31);
        if (!(done.load(std::memory_order_acquire) & bit)) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            done.fetch_or(bit, std::memory_order_release);
        }
        kern<<<grid, LAT::TX * TY, smem, s>>>(*map, a);
        return cudaGetLastError();
    }
}

template <typename LAT, typename R, int TY, int MODE, int SLOTS, bool TMA>
static cudaError_t launch_width(const Step3Args<R>& a, const CUtensorMap* map, dim3 grid, cudaStream_t s) {
    const bool narrow = (unsigned long long)a.P * LAT::Q < (1ULL << 32);
    return narrow ? launch_staged<LAT, R, TY, MODE, uint32_t, SLOTS, TMA>(a, map, grid, s)
                  : launch_staged<LAT, R, TY, MODE, unsigned long long, SLOTS, TMA>(a, map, grid, s);
}

// the staged variants a lattice offers: by copies in two or three slots on 32 x 8 (D3Q19) or
// 32 x 4 (D3Q27) tiles, and in FP32 by TMA (D3Q19 two or three slots on 32 x 6 tiles, 32 x 8
// with the correlated noise; D3Q27 two slots on 32 x 4)
template <typename LAT, typename R, int MODE>
static cudaError_t launch_mode3(const Step3Args<R>& a, const CUtensorMap* map, const Launch3& L, cudaStream_t s) {
    constexpr bool F32 = sizeof(R) == 4;
    if constexpr (LAT::Q == 19) {
        if (L.plain) {
            if constexpr (MODE == 0 || MODE == 1) {
                step3_kernel<R, MODE, 32, 8><<<L.grid, 256, 0, s>>>(a);
                return cudaGetLastError();
            }
            return cudaErrorInvalidValue;
        }
        if constexpr (F32) {
            // TMA: 32 x 6 tiles (four CTAs per SM in two slots), 32 x 8 with the correlated noise
            constexpr int TYT = MODE == 3 ? 8 : 6;
            if (L.tma)
                return L.slots == 2 ? launch_width<LAT, R, TYT, MODE, 2, true>(a, map, L.grid, s)
                                    : launch_width<LAT, R, TYT, MODE, 3, true>(a, map, L.grid, s);
        }
        return L.slots == 2 ? launch_width<LAT, R, 8, MODE, 2, false>(a, map, L.grid, s)
                            : launch_width<LAT, R, 8, MODE, 3, false>(a, map, L.grid, s);
    } else {
        if constexpr (F32) {
            if (L.tma) return launch_width<LAT, R, 4, MODE, 2, true>(a, map, L.grid, s);
        }
        return L.slots == 2 ? launch_width<LAT, R, 4, MODE, 2, false>(a, map, L.grid, s)
                            : launch_width<LAT, R, 4, MODE, 3, false>(a, map, L.grid, s);
    }
}

template <typename LAT, typename R>
cudaError_t launch_lattice(const Step3Args<R>& a, const CUtensorMap* map, const Launch3& L, cudaStream_t s) {
    if (L.kmode == 3) return launch_mode3<LAT, R, 3>(a, map, L, s);
    if (L.kmode == 4) return launch_mode3<LAT, R, 4>(a, map, L, s);
    return L.kmode ? launch_mode3<LAT, R, 1>(a, map, L, s) : launch_mode3<LAT, R, 0>(a, map, L, s);
}

// one translation unit per lattice instantiates these
extern template cudaError_t launch_lattice<Lat19, float>(const Step3Args<float>&, const CUtensorMap*, const Launch3&,
                                                         cudaStream_t);
extern template cudaError_t launch_lattice<Lat19, double>(const Step3Args<double>&, const CUtensorMap*,
                                                          const Launch3&, cudaStream_t);
extern template cudaError_t launch_lattice<Lat27, float>(const Step3Args<float>&, const CUtensorMap*, const Launch3&,
                                                         cudaStream_t);
extern template cudaError_t launch_lattice<Lat27, double>(const Step3Args<double>&, const CUtensorMap*,
                                                          const Launch3&, cudaStream_t);

}  // namespace lbf3
