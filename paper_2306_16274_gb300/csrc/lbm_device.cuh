// Device code of the fused non-orthogonal MRT pseudopotential step (sm_103a).
//
// Data layout: populations are structure-of-arrays, plane i holds f_bar_i for
// every cell, cell index (z*ny + y)*nx + x (x fastest), planes `plane` floats
// apart.  Streaming (Eq. e9) is done in place with the AA access pattern:
//   even step (parity 0): read f_i from slot i of the cell, write the
//     post-collision f*_i into slot ibar of the same cell;
//   odd step (parity 1): read f_i from slot ibar of x - e_i, write f*_i into
//     slot i of x + e_i.
// Each cell reads and writes the same set of locations, so the update needs no
// second copy.  Half-way bounce-back: on an odd step a link to a solid
// neighbour reads/writes the cell's own slot instead (f_i(x) <- slot i of x,
// f*_i -> slot ibar of x); an even step is local and needs no test.
//
// One-pass layout (optional, PARITY == 2 below): two copies; the copy being read holds the
// post-collision values of the previous step where they were computed, so population i of x is
// slot i of x - e_i (pull), and the step writes slot i of x in the other copy.
//
// Shifted FP16 store (optional): a slot holds h = f / rho_w - omega_i in half precision,
// rho_w being the density of the cell that wrote it, kept in FP32 in a density field.  The
// population f_i arriving at x was written by x - e_i (by x itself where that neighbour is
// solid), so the reader multiplies (omega_i + h) by that cell's density.  All arithmetic is FP32.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <climits>

#include "lbm_internal.h"
#include "transform_q19.cuh"
#include "transform_q27.cuh"

namespace lbm {

// ------------------------------------------------------------------ bounds-checked builds
// Compiled with LBM_BOUNDS_CHECK=1, every population, psi and ring access of the step kernels is
// checked against its array before it is made; an access outside is counted and redirected to
// element 0 (no trap), and the count is read by lbm_debug_bounds_violations.  Other builds
// compile the checks away.
#ifndef LBM_BOUNDS_CHECK
#define LBM_BOUNDS_CHECK 0
#endif
#if LBM_BOUNDS_CHECK
static __device__ unsigned long long lbm_bounds_count;
#endif
__device__ __forceinline__ uint32_t bounded(uint32_t off, unsigned long long limit) {
#if LBM_BOUNDS_CHECK
    if ((unsigned long long)off >= limit) {
        atomicAdd(&lbm_bounds_count, 1ull);
        return 0u;
    }
#endif
    (void)limit;
    return off;
}

// ------------------------------------------------------------------ lattice (Eq. e1)
__host__ __device__ constexpr int EX(int i) {
    constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int EY(int i) {
    constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int EZ(int i) {
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int OPP(int i) {
    constexpr int t[27] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15, 26, 25, 24, 23, 22, 21, 20, 19};
    return t[i];
}
// normalised weights w(|e|^2) = omega / c_s^2 of Eq. e15 for the active lattice
template <int Q>
__host__ __device__ constexpr float WN(int i) {
    return (EX(i) * EX(i) + EY(i) * EY(i) + EZ(i) * EZ(i)) == 1 ? (Q == 27 ? 2.0f / 9.0f : 1.0f / 6.0f)
         : (EX(i) * EX(i) + EY(i) * EY(i) + EZ(i) * EZ(i)) == 2 ? (Q == 27 ? 1.0f / 18.0f : 1.0f / 12.0f)
         : (EX(i) * EX(i) + EY(i) * EY(i) + EZ(i) * EZ(i)) == 3 ? 1.0f / 72.0f
         : 0.0f;
}

// lattice weights omega_i (Eq. e5; D3Q19: 1/3, 1/18, 1/36 of App. C)
template <int Q>
__host__ __device__ constexpr float OMEGA(int i) {
    return (EX(i) * EX(i) + EY(i) * EY(i) + EZ(i) * EZ(i)) == 0 ? (Q == 27 ? 8.0f / 27.0f : 1.0f / 3.0f)
         : (EX(i) * EX(i) + EY(i) * EY(i) + EZ(i) * EZ(i)) == 1 ? (Q == 27 ? 2.0f / 27.0f : 1.0f / 18.0f)
         : (EX(i) * EX(i) + EY(i) * EY(i) + EZ(i) * EZ(i)) == 2 ? (Q == 27 ? 1.0f / 54.0f : 1.0f / 36.0f)
         : 1.0f / 216.0f;
}

// population slot loads / stores in either storage type (FP32 values or FP16 shifted values)
// FP32 population slots are read once and written once per step; cache policy measured at 256^3
// (collide / density pass, ms): loads with a 256-byte L2 prefetch (the neighbouring tile's half of the
// line comes along) 0.4305 / 0.2056 on D3Q19 and 0.5875 / 0.2844 on D3Q27 against 0.4273 / 0.2077 and
// 0.5946 / 0.2884 with plain read-only loads; evict-first stores 0.4209 (D3Q19) and 0.5999 ms (D3Q27)
// against 0.4273 / 0.5946; loads bypassing L1 (.cg) no change; evict-first loads (.cs) 30 % slower.
// Kept: prefetching loads on both lattices, evict-first stores on D3Q19.
#ifndef LBM_LDPOP_HINT
#define LBM_LDPOP_HINT 2
#endif
#ifndef LBM_STPOP_CS
#define LBM_STPOP_CS (LBM_Q == 19)
#endif
__device__ __forceinline__ float ldpop(const float* p) {
#if LBM_LDPOP_HINT == 1
    return __ldcg(p);
#elif LBM_LDPOP_HINT == 2
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
#elif LBM_LDPOP_HINT == 3
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
#elif LBM_LDPOP_HINT == 4
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}
__device__ __forceinline__ float ldpop(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void stpop(float* p, float v) {
#if LBM_STPOP_CS
    __stcs(p, v);
#else
    *p = v;
#endif
}
__device__ __forceinline__ void stpop(__half* p, float v) { *p = __float2half_rn(v); }

template <int Q>
__device__ __forceinline__ void to_moments(const float (&f)[Q], float (&m)[Q]);
template <>
__device__ __forceinline__ void to_moments<19>(const float (&f)[19], float (&m)[19]) { moments_from_pops_q19(f, m); }
template <>
__device__ __forceinline__ void to_moments<27>(const float (&f)[27], float (&m)[27]) { moments_from_pops_q27(f, m); }
template <int Q>
__device__ __forceinline__ void to_pops(const float (&m)[Q], float (&f)[Q]);
template <>
__device__ __forceinline__ void to_pops<19>(const float (&m)[19], float (&f)[19]) { pops_from_moments_q19(m, f); }
template <>
__device__ __forceinline__ void to_pops<27>(const float (&m)[27], float (&f)[27]) { pops_from_moments_q27(m, f); }

// position of moment k of Eq. e11 in the lattice's moment vector (App. C keeps 0..15, 17, 18, 19)
template <int Q>
__host__ __device__ constexpr int MP(int k) { return (Q == 27 || k < 16) ? k : k - 1; }

// ------------------------------------------------------------------ neighbourhood of a cell
// idx / nb(): cell indices of the natural layout (fields, and populations unless paired);
// pidx / pnb(): population slot indices, which differ only in the x-paired FP16 layout.
struct Cell {
    int x, y, z;
    long long idx, pidx;
    int xo[3];        // x-1, x, x+1 wrapped (periodic)
    int pxo[3];       // their slot positions within a row (= xo unless paired)
    long long yo[3];  // (y+dy)*nx wrapped
    long long zo[3];  // (z+dz)*nx*ny wrapped
    __device__ __forceinline__ long long nb(int dx, int dy, int dz) const {
        return zo[dz + 1] + yo[dy + 1] + xo[dx + 1];
    }
    __device__ __forceinline__ long long pnb(int dx, int dy, int dz) const {
        return zo[dz + 1] + yo[dy + 1] + pxo[dx + 1];
    }
};

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// slot position of cell x within its row in the x-paired layout: word x mod hx, low half for
// x < hx, high half otherwise
__host__ __device__ __forceinline__ int pair_pos(int x, int hx) { return x < hx ? 2 * x : 2 * (x - hx) + 1; }

__device__ __forceinline__ Cell make_cell(const KParams& kp, int x, int y, int z) {
    Cell c;
    c.x = x;
    c.y = y;
    c.z = z;
    const long long nxy = (long long)kp.nx * kp.ny;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        c.xo[d + 1] = wrap1(x + d, kp.nx);
        c.pxo[d + 1] = kp.paired ? pair_pos(c.xo[d + 1], kp.hx) : c.xo[d + 1];
        c.yo[d + 1] = (long long)wrap1(y + d, kp.ny) * kp.nx;
        c.zo[d + 1] = (long long)wrap1(z + d, kp.nz) * nxy;
    }
    c.idx = z * nxy + (long long)y * kp.nx + x;
    c.pidx = z * nxy + (long long)y * kp.nx + c.pxo[1];
    return c;
}

// bit i set <=> x + e_i is solid (bit 0: the cell itself).  Walls are the planes
// just outside the domain on a wall axis; interior solids come from nbmask.
template <int Q>
__device__ __forceinline__ uint32_t solid_bits(const KParams& kp, const uint32_t* __restrict__ nbmask, const Cell& c) {
    uint32_t bits = nbmask ? __ldg(nbmask + c.idx) : 0u;
    const bool xl = kp.wall_x && c.x == 0, xh = kp.wall_x && c.x == kp.nx - 1;
    const bool yl = kp.wall_y && c.y == 0, yh = kp.wall_y && c.y == kp.ny - 1;
    const bool zl = kp.wall_z && c.z == 0, zh = kp.wall_z && c.z == kp.nz - 1;
    if (xl | xh | yl | yh | zl | zh) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const bool s = (EX(i) < 0 && xl) || (EX(i) > 0 && xh) || (EY(i) < 0 && yl) || (EY(i) > 0 && yh) ||
                           (EZ(i) < 0 && zl) || (EZ(i) > 0 && zh);
            bits |= s ? (1u << i) : 0u;
        }
    }
    return bits;
}

// ------------------------------------------------------------------ AA gather (raw slot values)
template <int Q, int PARITY, bool SOLIDS, class T>
__device__ __forceinline__ void gather(const KParams& kp, const T* __restrict__ f, const Cell& c, uint32_t bits,
                                       float (&p)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (PARITY == 2) {   // one-pass layout: pull from x - e_i
            p[i] = ldpop(f + i * kp.plane + c.pnb(-EX(i), -EY(i), -EZ(i)));
        } else if (PARITY == 0 || i == 0) {
            p[i] = ldpop(f + i * kp.plane + c.pidx);
        } else if (SOLIDS && ((bits >> OPP(i)) & 1u)) {
            p[i] = ldpop(f + i * kp.plane + c.pidx);   // reflected at the wall in the previous step
        } else {
            p[i] = ldpop(f + OPP(i) * kp.plane + c.pnb(-EX(i), -EY(i), -EZ(i)));
        }
    }
}

// Shifted FP16 store: slot values -> populations.  rs.at(dx, dy, dz) is the density of cell
// x + (dx, dy, dz) in the density field the slots were written with.
template <int Q, bool SOLIDS, class RS>
__device__ __forceinline__ void denorm(float (&p)[Q], uint32_t bits, const RS& rs) {
    const float self = rs.at(0, 0, 0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool own = i == 0 || (SOLIDS && ((bits >> OPP(i)) & 1u));
        const float r = own ? self : rs.at(-EX(i), -EY(i), -EZ(i));
        p[i] = (OMEGA<Q>(i) + p[i]) * r;
    }
}

// ... and populations -> slot values of a cell of density rho
template <int Q>
__device__ __forceinline__ void normalize(float (&p)[Q], float rho) {
    const float inv = 1.0f / rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) p[i] = p[i] * inv - OMEGA<Q>(i);
}

// density field lookups for denorm: three ring planes in shared memory, a 32-bit neighbourhood,
// or a 64-bit one
template <int SX = 1>
struct RsRingT {
    const float *pm, *p0, *pp;
    int sy;
    __device__ __forceinline__ float at(int dx, int dy, int dz) const {
        return (dz < 0 ? pm : (dz > 0 ? pp : p0))[SX * dx + dy * sy];
    }
};
using RsRing = RsRingT<1>;
struct RsCell {
    const float* r;
    const Cell& c;
    __device__ __forceinline__ float at(int dx, int dy, int dz) const { return __ldg(r + c.nb(dx, dy, dz)); }
};

// ------------------------------------------------------------------ equation of state -> psi
// ---- float-float arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, from the error-free transformations of Dekker (1971) and Knuth (TwoSum).
// The _rn intrinsics keep the compiler from fusing the error terms into other operations.
struct FF {
    float hi, lo;
};
// a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a + b exactly, any magnitudes
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = ff_two_sum(x.hi, y.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ FF ff_one_plus(FF x) {
    const FF s = ff_two_sum(1.0f, x.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
// products: the rounding error of hi * hi is exact with one FMA
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.hi, -p)));
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_mul(FF x, float f) {
    const float p = __fmul_rn(x.hi, f);
    return ff_fast_two_sum(p, __fmaf_rn(x.lo, f, __fmaf_rn(x.hi, f, -p)));
}
// x / y: a first quotient, then the exact remainder's quotient as its correction
__device__ __forceinline__ FF ff_div(FF x, FF y) {
    const float r = __frcp_rn(y.hi);
    const float q1 = __fmul_rn(x.hi, r);
    const FF rem = ff_add(x, ff_neg(ff_mul(y, q1)));
    return ff_fast_two_sum(q1, __fmul_rn(rem.hi, r));
}
__device__ __forceinline__ FF ff_of(float2 v) { return FF{v.x, v.y}; }

// (2/G)(p_EOS - rho c_s^2) of the Carnahan-Starling EOS in float-float.  On the liquid side the
// two terms of p_EOS nearly cancel (rho RT g(eta) ~ a rho^2 at coexistence), so a plain FP32
// evaluation keeps only ~14 good bits of p_EOS; here the result is ~44 bits good before it is
// rounded to float (written as rho (RT g(eta) / (1 - eta)^3 - a rho) - rho / 3, the same function).
__device__ __forceinline__ float cs_psi2_ff(const KParams& kp, float rho) {
    const FF eta = ff_mul(ff_of(kp.cs_b4_ff), rho);
    const FF om = ff_one_plus(ff_neg(eta));                                  // 1 - eta
    const FF om3 = ff_mul(ff_mul(om, om), om);
    const FF g = ff_one_plus(ff_mul(eta, ff_one_plus(ff_mul(eta, om))));    // 1 + eta + eta^2 - eta^3
    const FF br = ff_add(ff_div(ff_mul(ff_of(kp.cs_RT_ff), g), om3), ff_neg(ff_mul(ff_of(kp.cs_a_ff), rho)));
    const FF d = ff_add(ff_mul(br, rho), ff_neg(ff_mul(ff_of(kp.third_ff), rho)));
    return ff_mul(ff_of(kp.two_over_G_ff), d).hi;
}

// psi = sqrt(2 (p_EOS - rho c_s^2) / G) (Sec. II C).  The Carnahan-Starling liquid branch
// (rho >= psi_ext_rho) is evaluated in float-float arithmetic.
__device__ __forceinline__ float eval_psi(const KParams& kp, float rho, unsigned* status) {
    float psi2;
    if (kp.eos == 1) {
        if (rho >= kp.psi_ext_rho) {
            psi2 = cs_psi2_ff(kp, rho);
        } else {
            const float eta = kp.cs_b4 * rho;
            const float om = 1.0f - eta;
            const float p = rho * kp.cs_RT * (1.0f + eta * (1.0f + eta * (1.0f - eta))) / (om * om * om) -
                            kp.cs_a * rho * rho;
            psi2 = kp.two_over_G * (p - rho * (1.0f / 3.0f));
        }
    } else {
        float p;
        if (rho <= kp.pw_rho1) p = rho * kp.pw_tv;
        else if (rho <= kp.pw_rho2) p = kp.pw_p1 + (rho - kp.pw_rho1) * kp.pw_tm;
        else p = kp.pw_p2 + (rho - kp.pw_rho2) * kp.pw_tl;
        psi2 = kp.two_over_G * (p - rho * (1.0f / 3.0f));
    }
    if (!(psi2 >= 0.0f)) {
        atomicOr(status, ST_EOS_RANGE);
        psi2 = 0.0f;
    }
    return sqrtf(psi2);
}

// ------------------------------------------------------------------ psi stencil -> forces
struct Forces {
    float fx, fy, fz;        // F_int + F_ads (body force added later)
    float qxx, qyy, qzz, qxy, qxz, qyz;
    float s2;                // |S|^2, S = sum_i w_i psi(x + e_i) e_i  (|F_int|^2 / psi^2 = G^2 |S|^2)
};

// t points at psi(x) inside a tile with x stride 1, y stride sy, z stride sz.
template <int Q, bool SOLIDS>
__device__ __forceinline__ Forces stencil_forces(const KParams& kp, const float* t, int sy, int sz, uint32_t bits) {
    const float pc = t[0];
    float Sx = 0.f, Sy = 0.f, Sz = 0.f, Ax = 0.f, Ay = 0.f, Az = 0.f;
    float qxx = 0.f, qyy = 0.f, qzz = 0.f, qxy = 0.f, qxz = 0.f, qyz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        float pn = t[EX(i) + EY(i) * sy + EZ(i) * sz];
        if (SOLIDS && ((bits >> i) & 1u)) {
            pn = pc;   // neutral continuation at a solid neighbour; wetting enters through F_ads only
            Ax += WN<Q>(i) * EX(i);
            Ay += WN<Q>(i) * EY(i);
            Az += WN<Q>(i) * EZ(i);
        }
        const float wp = WN<Q>(i) * pn;
        if (EX(i)) Sx += EX(i) > 0 ? wp : -wp;
        if (EY(i)) Sy += EY(i) > 0 ? wp : -wp;
        if (EZ(i)) Sz += EZ(i) > 0 ? wp : -wp;
        const float wd = WN<Q>(i) * (pn - pc);
        if (EX(i)) qxx += wd;
        if (EY(i)) qyy += wd;
        if (EZ(i)) qzz += wd;
        if (EX(i) && EY(i)) qxy += (EX(i) * EY(i) > 0) ? wd : -wd;
        if (EX(i) && EZ(i)) qxz += (EX(i) * EZ(i) > 0) ? wd : -wd;
        if (EY(i) && EZ(i)) qyz += (EY(i) * EZ(i) > 0) ? wd : -wd;
    }
    Forces F;
    const float gp = -kp.G * pc;
    const float ga = -kp.G_ads * pc * pc;
    F.fx = gp * Sx + ga * Ax;
    F.fy = gp * Sy + ga * Ay;
    F.fz = gp * Sz + ga * Az;
    const float kq = kp.kappa_G_half * pc;
    F.qxx = kq * qxx;
    F.qyy = kq * qyy;
    F.qzz = kq * qzz;
    F.qxy = kq * qxy;
    F.qxz = kq * qxz;
    F.qyz = kq * qyz;
    F.s2 = Sx * Sx + Sy * Sy + Sz * Sz;
    return F;
}

// ------------------------------------------------------------------ collision in moment space
// m_bar* = m_bar - S (m_bar - m^eq) + (I - S/2) F~'   (Eq. e8), m^eq of Eq. e13,
// F~ of Eq. e14 with the Eq. e17 modifications.  The conserved moments are
// written in closed form: m*_0 = m_0, m*_{1..3} = m_{1..3} + F (exactly what
// Eq. e8 gives once rho u = m_{1..3} + F/2).
template <int Q>
__device__ __forceinline__ void collide(const KParams& kp, float (&f)[Q], const Forces& Fo, float& rho_out,
                                        float& ux_out, float& uy_out, float& uz_out) {
    float m[Q];
    to_moments<Q>(f, m);
    const float rho = m[0];
    const float inv_rho = 1.0f / rho;
    const float Fx = Fo.fx + rho * kp.gx;
    const float Fy = Fo.fy + rho * kp.gy;
    const float Fz = Fo.fz + rho * kp.gz;
    const float ux = (m[1] + 0.5f * Fx) * inv_rho;
    const float uy = (m[2] + 0.5f * Fy) * inv_rho;
    const float uz = (m[3] + 0.5f * Fz) * inv_rho;
    rho_out = rho;
    ux_out = ux;
    uy_out = uy;
    uz_out = uz;

    float s_nu = kp.s[2], c_nu = kp.c[2], inv_tnu = kp.inv_tnu;
    if (kp.variable_nu) {   // Sec. IV A: nu(rho), nu = (1/s_nu - 1/2) c_s^2
        const float nu = kp.nu_v + kp.dnu_drho * (rho - kp.rho_v);
        s_nu = 1.0f / (3.0f * nu + 0.5f);
        c_nu = 1.0f - 0.5f * s_nu;
        inv_tnu = 1.0f / (3.0f * nu);
    }
    const float cs2 = 1.0f / 3.0f, cs4 = 1.0f / 9.0f, cs6 = 1.0f / 27.0f;
    const float uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    const float ru_x = rho * ux, ru_y = rho * uy, ru_z = rho * uz;
    const float Fxux = Fx * ux, Fyuy = Fy * uy, Fzuz = Fz * uz;
    const float Fu = Fxux + Fyuy + Fzuz;
    const float Fxy = Fx * uy + Fy * ux, Fxz = Fx * uz + Fz * ux, Fyz = Fy * uz + Fz * uy;

#define RELAX(k, meq, Ft, s, c) m[MP<Q>(k)] += (s) * ((meq) - m[MP<Q>(k)]) + (c) * (Ft)
    m[1] += Fx;
    m[2] += Fy;
    m[3] += Fz;
    RELAX(4, ru_x * uy, Fxy - Fo.qxy * inv_tnu, s_nu, c_nu);
    RELAX(5, ru_x * uz, Fxz - Fo.qxz * inv_tnu, s_nu, c_nu);
    RELAX(6, ru_y * uz, Fyz - Fo.qyz * inv_tnu, s_nu, c_nu);
    RELAX(7, rho * (1.0f + uxx + uyy + uzz),
          2.0f * Fu + kp.sigma_coef * Fo.s2 + kp.q7_coef * (Fo.qxx + Fo.qyy + Fo.qzz), kp.s[3], kp.c[3]);
    RELAX(8, rho * (uxx - uyy), 2.0f * (Fxux - Fyuy) - (Fo.qxx - Fo.qyy) * inv_tnu, s_nu, c_nu);
    RELAX(9, rho * (uxx - uzz), 2.0f * (Fxux - Fzuz) - (Fo.qxx - Fo.qzz) * inv_tnu, s_nu, c_nu);
    RELAX(10, cs2 * ru_x, cs2 * Fx, kp.s[4], kp.c[4]);
    RELAX(11, cs2 * ru_x, cs2 * Fx, kp.s[4], kp.c[4]);
    RELAX(12, cs2 * ru_y, cs2 * Fy, kp.s[4], kp.c[4]);
    RELAX(13, cs2 * ru_z, cs2 * Fz, kp.s[4], kp.c[4]);
    RELAX(14, cs2 * ru_y, cs2 * Fy, kp.s[4], kp.c[4]);
    RELAX(15, cs2 * ru_z, cs2 * Fz, kp.s[4], kp.c[4]);
    if (Q == 27) RELAX(16, 0.0f, 0.0f, kp.s[5], kp.c[5]);
    RELAX(17, cs2 * rho * (cs2 + uxx + uyy), 2.0f * cs2 * (Fxux + Fyuy), kp.s[6], kp.c[6]);
    RELAX(18, cs2 * rho * (cs2 + uxx + uzz), 2.0f * cs2 * (Fxux + Fzuz), kp.s[6], kp.c[6]);
    RELAX(19, cs2 * rho * (cs2 + uyy + uzz), 2.0f * cs2 * (Fyuy + Fzuz), kp.s[6], kp.c[6]);
    if (Q == 27) {
        RELAX(20, cs2 * ru_y * uz, cs2 * Fyz, kp.s[7], kp.c[7]);
        RELAX(21, cs2 * ru_x * uz, cs2 * Fxz, kp.s[7], kp.c[7]);
        RELAX(22, cs2 * ru_x * uy, cs2 * Fxy, kp.s[7], kp.c[7]);
        RELAX(23, cs4 * ru_x, cs4 * Fx, kp.s[8], kp.c[8]);
        RELAX(24, cs4 * ru_y, cs4 * Fy, kp.s[8], kp.c[8]);
        RELAX(25, cs4 * ru_z, cs4 * Fz, kp.s[8], kp.c[8]);
        RELAX(26, cs4 * rho * (uxx + uyy + uzz) + cs6 * rho, 2.0f * cs4 * Fu, kp.s[9], kp.c[9]);
    }
#undef RELAX
    to_pops<Q>(m, f);
}

// ------------------------------------------------------------------ 32-bit neighbourhood (z-marching kernels)
// Offsets are cell indices (< 2^31); addresses are formed from the per-plane base
// pointers kp.fq[i], which live in the kernel-parameter constant bank.
struct Off32 {
    uint32_t c;       // the cell
    uint32_t xo[3];   // x-1, x, x+1 wrapped
    uint32_t yo[3];   // rows y-1, y, y+1 wrapped, times nx
    uint32_t zo[3];   // planes z-1, z, z+1 wrapped, times nx*ny
    __device__ __forceinline__ uint32_t nb(int dx, int dy, int dz) const { return zo[dz + 1] + yo[dy + 1] + xo[dx + 1]; }
};

// Geometry accessors: the domain's extents and wall flags, read from the kernel parameters
// (single-domain launches) or from the block's member record in shared memory (multi-domain).
struct KGeom {
    const KParams& k;
    __device__ __forceinline__ int nx() const { return k.nx; }
    __device__ __forceinline__ int ny() const { return k.ny; }
    __device__ __forceinline__ int nz() const { return k.nz; }
    __device__ __forceinline__ int wall_x() const { return k.wall_x; }
    __device__ __forceinline__ int wall_y() const { return k.wall_y; }
    __device__ __forceinline__ int wall_z() const { return k.wall_z; }
};
struct DGeom {
    const BatchDom& d;
    __device__ __forceinline__ int nx() const { return d.nx; }
    __device__ __forceinline__ int ny() const { return d.ny; }
    __device__ __forceinline__ int nz() const { return d.nz; }
    __device__ __forceinline__ int wall_x() const { return d.wall_x; }
    __device__ __forceinline__ int wall_y() const { return d.wall_y; }
    __device__ __forceinline__ int wall_z() const { return d.wall_z; }
};

template <int Q, class GM>
__device__ __forceinline__ uint32_t solid_bits32(const GM& g, const uint32_t* __restrict__ nbmask, uint32_t c,
                                                 int x, int y, int z) {
    uint32_t bits = nbmask ? __ldg(nbmask + c) : 0u;
    const bool xl = g.wall_x() && x == 0, xh = g.wall_x() && x == g.nx() - 1;
    const bool yl = g.wall_y() && y == 0, yh = g.wall_y() && y == g.ny() - 1;
    const bool zl = g.wall_z() && z == 0, zh = g.wall_z() && z == g.nz() - 1;
    if (xl | xh | yl | yh | zl | zh) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const bool s = (EX(i) < 0 && xl) || (EX(i) > 0 && xh) || (EY(i) < 0 && yl) || (EY(i) > 0 && yh) ||
                           (EZ(i) < 0 && zl) || (EZ(i) > 0 && zh);
            bits |= s ? (1u << i) : 0u;
        }
    }
    return bits;
}

// Address of cell offset `off` in population plane i: per-plane base pointers from the kernel
// parameters (constant bank, free operands) for single-domain launches (T = float, or __half for
// the shifted FP16 store) ...
template <class T>
struct PlanePtrsT {
    const KParams& kp;
    __device__ __forceinline__ T* ptr(int i, uint32_t off) const {
#if LBM_BOUNDS_CHECK
        if (i < 0 || i >= 27 || !kp.fq[i]) {
            atomicAdd(&lbm_bounds_count, 1ull);
            i = 0;
        }
#endif
        return reinterpret_cast<T*>(kp.fq[i]) + bounded(off, (unsigned long long)kp.ncell);
    }
};
using PlanePtrs = PlanePtrsT<float>;
// ... or, for multi-domain launches, one base pointer and a 32-bit plane stride: the whole
// index i * plane + off stays in 32 bits (a member's Q planes hold < 2^32 floats), so each access
// costs one integer multiply-add and one wide address computation.
struct PlaneIdx32 {
    const float* base;
    uint32_t plane;
    __device__ __forceinline__ float* ptr(int i, uint32_t off) const {
        return const_cast<float*>(base) + (uint32_t)((uint32_t)i * plane + bounded(off, plane));
    }
};
// ... or the member record itself: the plane stride is read from the (constant-bank) record at each
// use instead of being held in a register, which leaves the multi-domain collide kernel registers
// for the psi-ring prefetch.
struct DomPlanes {
    const BatchDom& d;
    __device__ __forceinline__ float* ptr(int i, uint32_t off) const {
        return d.base + (uint32_t)((uint32_t)i * (uint32_t)d.plane +
                                   bounded(off, (unsigned long long)d.nx * d.ny * d.nz));
    }
};

struct RsOff32 {
    const float* r;
    const Off32& o;
    __device__ __forceinline__ float at(int dx, int dy, int dz) const { return __ldg(r + o.nb(dx, dy, dz)); }
};

template <int Q, int PARITY, bool SOLIDS, class A>
__device__ __forceinline__ void gather32(const A& a, const Off32& o, uint32_t bits, float (&p)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (PARITY == 2) {   // one-pass layout: pull from x - e_i
            p[i] = ldpop(a.ptr(i, o.nb(-EX(i), -EY(i), -EZ(i))));
        } else if (PARITY == 0 || i == 0) {
            p[i] = ldpop(a.ptr(i, o.c));
        } else if (SOLIDS && ((bits >> OPP(i)) & 1u)) {
            p[i] = ldpop(a.ptr(i, o.c));
        } else {
            p[i] = ldpop(a.ptr(OPP(i), o.nb(-EX(i), -EY(i), -EZ(i))));
        }
    }
}

template <int Q, int PARITY, bool SOLIDS, class A>
__device__ __forceinline__ void store32(const A& a, const Off32& o, uint32_t bits, const float (&p)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (PARITY == 0 || i == 0) {
            stpop(a.ptr(OPP(i), o.c), p[i]);
        } else if (SOLIDS && ((bits >> i) & 1u)) {
            stpop(a.ptr(OPP(i), o.c), p[i]);
        } else {
            stpop(a.ptr(i, o.nb(EX(i), EY(i), EZ(i))), p[i]);
        }
    }
}

// Forces from three psi planes (z-1, z, z+1); each pointer addresses psi(x) within its plane,
// x stride SX and y stride sy.
template <int Q, bool SOLIDS, int SX = 1>
__device__ __forceinline__ Forces stencil_forces3(const KParams& kp, const float* pm, const float* p0, const float* pp,
                                                  int sy, uint32_t bits) {
    const float pc = p0[0];
    float Sx = 0.f, Sy = 0.f, Sz = 0.f, Ax = 0.f, Ay = 0.f, Az = 0.f;
    float qxx = 0.f, qyy = 0.f, qzz = 0.f, qxy = 0.f, qxz = 0.f, qyz = 0.f;
    float pn[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float* pl = EZ(i) < 0 ? pm : (EZ(i) > 0 ? pp : p0);
        pn[i] = pl[SX * EX(i) + EY(i) * sy];
        if (SOLIDS && ((bits >> i) & 1u)) {   // a solid neighbour: psi(x) there, and F_ads
            pn[i] = pc;
            Ax += WN<Q>(i) * EX(i);
            Ay += WN<Q>(i) * EY(i);
            Az += WN<Q>(i) * EZ(i);
        }
    }
    // opposite links together: w e (psi_i - psi_ibar) for F_int, w e e (psi_i + psi_ibar - 2 psi(x))
    // for Q (e_ibar = -e_i, equal weights)
    const float pc2 = 2.0f * pc;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (OPP(i) < i) continue;
        const float a = pn[i] - pn[OPP(i)];
        const float b = (pn[i] + pn[OPP(i)]) - pc2;
        const float w = WN<Q>(i);
        if (EX(i)) Sx += (EX(i) > 0 ? w : -w) * a;
        if (EY(i)) Sy += (EY(i) > 0 ? w : -w) * a;
        if (EZ(i)) Sz += (EZ(i) > 0 ? w : -w) * a;
        if (EX(i)) qxx += w * b;
        if (EY(i)) qyy += w * b;
        if (EZ(i)) qzz += w * b;
        if (EX(i) && EY(i)) qxy += (EX(i) * EY(i) > 0 ? w : -w) * b;
        if (EX(i) && EZ(i)) qxz += (EX(i) * EZ(i) > 0 ? w : -w) * b;
        if (EY(i) && EZ(i)) qyz += (EY(i) * EZ(i) > 0 ? w : -w) * b;
    }
    Forces F;
    const float gp = -kp.G * pc;
    const float ga = -kp.G_ads * pc * pc;
    F.fx = gp * Sx + ga * Ax;
    F.fy = gp * Sy + ga * Ay;
    F.fz = gp * Sz + ga * Az;
    const float kq = kp.kappa_G_half * pc;
    F.qxx = kq * qxx;
    F.qyy = kq * qyy;
    F.qzz = kq * qzz;
    F.qxy = kq * qxy;
    F.qxz = kq * qxz;
    F.qyz = kq * qyz;
    F.s2 = Sx * Sx + Sy * Sy + Sz * Sz;
    return F;
}

// ------------------------------------------------------------------ psi tile in shared memory
// Block of BX x BY x BZ cells; the tile holds psi for the block plus a one-cell
// halo (periodic wrap; 0 beyond a wall, where the solid bits take over).
template <int BX, int BY, int BZ>
struct PsiTile {
    static constexpr int TX = BX + 2, TY = BY + 2, TZ = BZ + 2, SIZE = TX * TY * TZ;
    float v[SIZE];

    __device__ __forceinline__ void load(const KParams& kp, const float* __restrict__ psi, int x0, int y0, int z0,
                                         int tid) {
        const long long nxy = (long long)kp.nx * kp.ny;
        for (int k = tid; k < SIZE; k += BX * BY * BZ) {
            const int tx = k % TX, ty = (k / TX) % TY, tz = k / (TX * TY);
            int gx = x0 - 1 + tx, gy = y0 - 1 + ty, gz = z0 - 1 + tz;
            bool ok = true;
            if (gx < 0) { ok &= !kp.wall_x; gx += kp.nx; } else if (gx >= kp.nx) { ok &= !kp.wall_x; gx -= kp.nx; }
            if (gy < 0) { ok &= !kp.wall_y; gy += kp.ny; } else if (gy >= kp.ny) { ok &= !kp.wall_y; gy -= kp.ny; }
            if (gz < 0) { ok &= !kp.wall_z; gz += kp.nz; } else if (gz >= kp.nz) { ok &= !kp.wall_z; gz -= kp.nz; }
            // one wrap suffices for every cell an active thread reads; anything still outside is unused
            ok = ok && gx >= 0 && gx < kp.nx && gy >= 0 && gy < kp.ny && gz >= 0 && gz < kp.nz;
            v[k] = ok ? __ldg(psi + gz * nxy + (long long)gy * kp.nx + gx) : 0.0f;
        }
    }
    __device__ __forceinline__ const float* at(int lx, int ly, int lz) const {
        return v + (lz + 1) * TX * TY + (ly + 1) * TX + (lx + 1);
    }
};

}  // namespace lbm
