// Kernels of one lattice; included by kernels_q19.cu / kernels_q27.cu with LBM_Q set.
#pragma once

#include <cmath>
#include <type_traits>

#include "lbm_device.cuh"

#ifndef LBM_Q
#error "define LBM_Q (19 or 27) before including kernels_impl.cuh"
#endif

namespace lbm {
namespace {

constexpr int Q = LBM_Q;

// ---- density + psi pass (Sec. II A, Sec. II C): one thread per cell, x fastest
constexpr int PSI_BX = 32, PSI_BY = 4;

// Shape of a tile: BX x BY cells in (x, y), one thread each; the z-marching collide kernels keep a
// psi ring plane of it with a one-cell halo.  The single-domain kernels use 32 x 4 (ZmTile); the
// multi-domain kernels any shape of BATCH_SHAPES, chosen per group by lbm_batch_tune.
template <int BX_, int BY_>
struct TileShape {
    static constexpr int BX = BX_, BY = BY_, NT = BX * BY;
    static constexpr int RX = BX + 2, RY = BY + 2, RP = RX * RY;
    static constexpr int SLOTS = (RP + NT - 1) / NT;   // ring loads per thread per plane
};
template <int S>
using BatchTileShape = TileShape<BATCH_SHAPES[S].bx, BATCH_SHAPES[S].by>;
template <int S>
constexpr int batch_minb() { return LBM_Q == 19 ? BATCH_SHAPES[S].minb19 : BATCH_SHAPES[S].minb27; }

// cells (x, y, z) for z in [z0, z1) of one column: pull the populations (AA phase PARITY),
// rho = sum f, psi from the equation of state.  F16: the slots hold the shifted FP16 store,
// read with the densities rsrc they were written with; the new densities go to rdst.
template <int PARITY, bool SOLIDS, bool F16, class GM, class A>
__device__ __forceinline__ void psi_column(const KParams& kp, const GM& g, const A& addr, float* __restrict__ psi,
                                           const uint32_t* __restrict__ nbmask, unsigned* status, int x, int y,
                                           int z0, int z1, const float* __restrict__ rsrc, float* __restrict__ rdst) {
    const int nx = g.nx(), ny = g.ny(), nz = g.nz();
    if (x >= nx || y >= ny) return;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
    Off32 o;
    o.xo[0] = (uint32_t)wrap1(x - 1, nx);
    o.xo[1] = (uint32_t)x;
    o.xo[2] = (uint32_t)wrap1(x + 1, nx);
    o.yo[0] = (uint32_t)wrap1(y - 1, ny) * (uint32_t)nx;
    o.yo[1] = (uint32_t)y * (uint32_t)nx;
    o.yo[2] = (uint32_t)wrap1(y + 1, ny) * (uint32_t)nx;
    for (int z = z0; z < z1; ++z) {
        o.zo[0] = (uint32_t)wrap1(z - 1, nz) * nxy;
        o.zo[1] = (uint32_t)z * nxy;
        o.zo[2] = (uint32_t)wrap1(z + 1, nz) * nxy;
        o.c = o.zo[1] + o.yo[1] + o.xo[1];
        const uint32_t bits = SOLIDS ? solid_bits32<Q>(g, nbmask, o.c, x, y, z) : 0u;
        if (bits & 1u) {
            if (kp.multiphase) psi[bounded(o.c, (unsigned long long)nxy * nz)] = 0.0f;
            if (F16) rdst[o.c] = 1.0f;
            continue;
        }
        float p[Q];
        gather32<Q, PARITY, SOLIDS>(addr, o, bits, p);
        if (F16) denorm<Q, SOLIDS>(p, bits, RsOff32{rsrc, o});
        float rho = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) rho += p[i];
        if (F16) rdst[o.c] = rho;
        if (kp.multiphase) psi[bounded(o.c, (unsigned long long)nxy * nz)] = eval_psi(kp, rho, status);
    }
}

template <int PARITY, bool SOLIDS, bool F16>
__global__ void __launch_bounds__(PSI_BX * PSI_BY) psi_kernel(KParams kp, float* __restrict__ psi,
                                                            const uint32_t* __restrict__ nbmask, unsigned* status,
                                                            const float* __restrict__ rsrc,
                                                            float* __restrict__ rdst) {
    const KGeom g{kp};
    const PlanePtrsT<typename std::conditional<F16, __half, float>::type> addr{kp};
    psi_column<PARITY, SOLIDS, F16>(kp, g, addr, psi, nbmask, status, blockIdx.x * PSI_BX + threadIdx.x,
                                    blockIdx.y * PSI_BY + threadIdx.y, blockIdx.z, blockIdx.z + 1, rsrc, rdst);
}


// multi-domain density + psi pass: one block per tile (of shape S) of any member of the launch's
// table; physics by value
template <int PARITY, bool SOLIDS, int S>
__global__ void __launch_bounds__(BatchTileShape<S>::NT) psi_batch_kernel(const KParams phys,
                                                                       const __grid_constant__ BatchDomTable tab,
                                                                       const BatchTile* __restrict__ tiles) {
    const BatchTile t = tiles[blockIdx.x];
    const BatchDom& m = tab.d[t.d];
    const DGeom g{m};
    const PlaneIdx32 addr{m.base, (uint32_t)m.plane};
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int w = t.narrow ? BATCH_NARROW_BX : (int)blockDim.x;   // a narrow tile: 16 cells wide
    psi_column<PARITY, SOLIDS, false>(phys, g, addr, m.psi, m.nbmask, m.status, t.x0 + tid % w, t.y0 + tid / w, t.z0,
                                      min(t.z0 + t.zc, m.nz), nullptr, nullptr);
}

// multi-domain density + psi pass over runs of whole planes (cells without solid handling): thread k
// of a block takes cells begin + k, begin + k + RUN_NT, ... of its run, so rows of any length pack
// the warps densely.  Per cell the arithmetic and its order are psi_column's.
constexpr int RUN_NT = 256;
__device__ __forceinline__ uint32_t div_by_magic(uint32_t n, uint32_t m, int s) {
    return (uint32_t)(((unsigned long long)m * n) >> s);
}
template <int PARITY>
__global__ void __launch_bounds__(RUN_NT) psi_run_kernel(const KParams phys, const __grid_constant__ BatchDomTable tab,
                                                         const BatchRun* __restrict__ runs) {
    const BatchRun r = runs[blockIdx.x];
    const BatchDom& m = tab.d[r.d];
    const PlaneIdx32 addr{m.base, (uint32_t)m.plane};
    const uint32_t nx = (uint32_t)m.nx, ny = (uint32_t)m.ny, nz = (uint32_t)m.nz, nxy = nx * ny;
    for (uint32_t c = r.begin + threadIdx.x; c < r.end; c += RUN_NT) {
        const uint32_t row = div_by_magic(c, m.mx, m.sx), x = c - row * nx;
        const uint32_t z = div_by_magic(row, m.my, m.sy), y = row - z * ny;
        Off32 o;
        o.xo[0] = (uint32_t)wrap1((int)x - 1, (int)nx);
        o.xo[1] = x;
        o.xo[2] = (uint32_t)wrap1((int)x + 1, (int)nx);
        o.yo[0] = (uint32_t)wrap1((int)y - 1, (int)ny) * nx;
        o.yo[1] = y * nx;
        o.yo[2] = (uint32_t)wrap1((int)y + 1, (int)ny) * nx;
        o.zo[0] = (uint32_t)wrap1((int)z - 1, (int)nz) * nxy;
        o.zo[1] = z * nxy;
        o.zo[2] = (uint32_t)wrap1((int)z + 1, (int)nz) * nxy;
        o.c = c;
        float p[Q];
        gather32<Q, PARITY, false>(addr, o, 0u, p);
        float rho = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) rho += p[i];
        m.psi[bounded(c, (unsigned long long)nxy * nz)] = eval_psi(phys, rho, m.status);
    }
}

// ---- fused collide-stream pass: psi tile -> forces -> gather -> moments -> relax -> M^-1 -> store
// Tiles of 32 x ZM_BY cells in (x, y) march through a chunk of z planes.  psi planes
// z-1, z, z+1 (with a one-cell x/y halo) sit in a four-slot shared-memory ring, so
// each plane is read once per tile and one barrier per plane suffices.  (Staging the
// populations through shared memory with cp.async measured slower: it doubles the
// load/store instructions of an issue-bound kernel.)
constexpr int CS_BX = 32, CS_BY = 4, CS_BZ = 2;        // 3D tile shape of the moments kernel
// tile height and blocks per SM (register caps 73 for D3Q19, 102 for D3Q27), with the next
// plane's populations prefetched into registers: the best of measured sweeps over tile
// height 2/4/8, 3-16 blocks per SM, prefetch on/off and the shared-memory carveout on 256^3
#ifndef LBM_ZM_BY
#define LBM_ZM_BY 4
#endif
#ifndef LBM_ZM_MINB19
#define LBM_ZM_MINB19 7
#endif
#ifndef LBM_ZM_MINB27
#define LBM_ZM_MINB27 5
#endif
constexpr int ZM_BX = 32, ZM_BY = LBM_ZM_BY, ZM_MINB = LBM_Q == 19 ? LBM_ZM_MINB19 : LBM_ZM_MINB27;

using ZmTile = TileShape<ZM_BX, ZM_BY>;

// plane offsets of z in a 32-bit neighbourhood
__device__ __forceinline__ void set_plane(Off32& o, int z, int nz, uint32_t nxy) {
    o.zo[0] = (uint32_t)wrap1(z - 1, nz) * nxy;
    o.zo[1] = (uint32_t)z * nxy;
    o.zo[2] = (uint32_t)wrap1(z + 1, nz) * nxy;
    o.c = o.zo[1] + o.yo[1] + o.xo[1];
}

// psi plane zz (wrapped, or zeros beyond a wall) into one ring slot; each thread loads its
// TS::SLOTS entries, whose x/y offsets are fixed for the whole march.
template <class TS>
__device__ __forceinline__ void load_psi_plane(float* slot, const float* __restrict__ psi, int zz, int nz, int wall_z,
                                               uint32_t nxy, const uint32_t (&goff)[TS::SLOTS],
                                               const bool (&gok)[TS::SLOTS], int tid) {
    bool zok = true;
    if (zz < 0) { zok = !wall_z; zz += nz; } else if (zz >= nz) { zok = !wall_z; zz -= nz; }
    const uint32_t zb = (uint32_t)zz * nxy;
#pragma unroll
    for (int s = 0; s < TS::SLOTS; ++s) {
        const int k = tid + s * TS::NT;
        if (k < TS::RP) slot[k] = (zok && gok[s]) ? __ldg(psi + bounded(zb + goff[s], (unsigned long long)nxy * nz)) : 0.0f;
    }
}

// the same plane in two halves: the loads into registers, then (an iteration later) the stores
// into the ring slot, so that the loads' latency is spent on a plane's collision
template <class TS>
__device__ __forceinline__ void fetch_psi_plane(float (&v)[TS::SLOTS], const float* __restrict__ psi, int zz, int nz,
                                                int wall_z, uint32_t nxy, const uint32_t (&goff)[TS::SLOTS],
                                                const bool (&gok)[TS::SLOTS], int tid) {
    bool zok = true;
    if (zz < 0) { zok = !wall_z; zz += nz; } else if (zz >= nz) { zok = !wall_z; zz -= nz; }
    const uint32_t zb = (uint32_t)zz * nxy;
#pragma unroll
    for (int s = 0; s < TS::SLOTS; ++s) {
        const int k = tid + s * TS::NT;
        v[s] = (k < TS::RP && zok && gok[s]) ? __ldg(psi + bounded(zb + goff[s], (unsigned long long)nxy * nz)) : 0.0f;
    }
}
template <class TS>
__device__ __forceinline__ void put_psi_plane(float* slot, const float (&v)[TS::SLOTS], int tid) {
#pragma unroll
    for (int s = 0; s < TS::SLOTS; ++s) {
        const int k = tid + s * TS::NT;
        if (k < TS::RP) slot[k] = v[s];
    }
}

#ifndef LBM_ZM_PREFETCH
#define LBM_ZM_PREFETCH 1
#endif

// One tile: cells [x0, x0+TS::BX) x [y0, y0+TS::BY) marching through planes [z0, z0+zchunk); `addr`
// locates population planes.  F16 (shifted FP16 store): the densities the slots were written
// with (rsrc) follow the march in a second shared ring `rring`; outputs are written relative
// to the cell's current density rown.
// PSI_PF: the psi (and FP16 density) ring planes are loaded into registers one plane ahead and
// stored into the ring at the next plane (all but the multi-domain kernels' solid tiles, which
// have no registers to spare and load each plane just before its barrier).
template <class TS, int PARITY, bool SOLIDS, bool MULTIPHASE, bool F16, bool PSI_PF, class GM, class A,
          bool FLAT = false>
__device__ __forceinline__ void collide_tile(const KParams& kp, const GM& g, const A& addr, const float* __restrict__ psi,
                                             const uint32_t* __restrict__ nbmask, unsigned* status, int x0, int y0,
                                             int z0, int zchunk, int zmax, float (*ring)[TS::RP], float (*rring)[TS::RP],
                                             const float* __restrict__ rsrc, const float* __restrict__ rown) {
    // FLAT: the block has another shape with as many threads (a narrow multi-domain tile); its threads
    // take the tile's cells in row-major order
    const int tid = FLAT ? (int)(threadIdx.x + blockDim.x * threadIdx.y) : (int)(threadIdx.x + TS::BX * threadIdx.y);
    const int tx = FLAT ? tid % TS::BX : (int)threadIdx.x, ty = FLAT ? tid / TS::BX : (int)threadIdx.y;
    const int x = x0 + tx, y = y0 + ty;
    const int nx = g.nx(), ny = g.ny(), nz = g.nz();
    const bool act_xy = x < nx && y < ny;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
    const int zend = min(z0 + zchunk, zmax);

    uint32_t goff[TS::SLOTS];
    bool gok[TS::SLOTS];
#pragma unroll
    for (int s = 0; s < TS::SLOTS; ++s) {
        const int k = tid + s * TS::NT;
        int gx = x0 - 1 + k % TS::RX, gy = y0 - 1 + k / TS::RX;
        bool ok = k < TS::RP;
        if (gx < 0) { ok &= !g.wall_x(); gx += nx; } else if (gx >= nx) { ok &= !g.wall_x(); gx -= nx; }
        if (gy < 0) { ok &= !g.wall_y(); gy += ny; } else if (gy >= ny) { ok &= !g.wall_y(); gy -= ny; }
        ok = ok && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        gok[s] = ok;
        goff[s] = ok ? (uint32_t)gy * (uint32_t)nx + (uint32_t)gx : 0u;
    }

    Off32 o;
    o.xo[0] = (uint32_t)wrap1(x - 1, nx);
    o.xo[1] = (uint32_t)x;
    o.xo[2] = (uint32_t)wrap1(x + 1, nx);
    o.yo[0] = (uint32_t)wrap1(y - 1, ny) * (uint32_t)nx;
    o.yo[1] = (uint32_t)y * (uint32_t)nx;
    o.yo[2] = (uint32_t)wrap1(y + 1, ny) * (uint32_t)nx;

#if LBM_ZM_PREFETCH
    // populations of the first plane, then of plane z+1 while plane z is computed; the first
    // plane's loads are issued before the ring's first planes are loaded and stored, so that the
    // chunk's start-up waits for one round trip instead of two
    float pn[Q];
    uint32_t bits_n = 0u;
    if (act_xy) {
        set_plane(o, z0, nz, nxy);
        bits_n = SOLIDS ? solid_bits32<Q>(g, nbmask, o.c, x, y, z0) : 0u;
        if (!(bits_n & 1u)) gather32<Q, PARITY, SOLIDS>(addr, o, bits_n, pn);
    }
#endif
    float pv[TS::SLOTS], rv[TS::SLOTS];
    if (PSI_PF && MULTIPHASE) fetch_psi_plane<TS>(pv, psi, z0 + 1, nz, g.wall_z(), nxy, goff, gok, tid);
    if (PSI_PF && F16) fetch_psi_plane<TS>(rv, rsrc, z0 + 1, nz, g.wall_z(), nxy, goff, gok, tid);
    if (MULTIPHASE) {
        load_psi_plane<TS>(ring[0], psi, z0 - 1, nz, g.wall_z(), nxy, goff, gok, tid);
        load_psi_plane<TS>(ring[1], psi, z0, nz, g.wall_z(), nxy, goff, gok, tid);
    }
    if (F16) {
        load_psi_plane<TS>(rring[0], rsrc, z0 - 1, nz, g.wall_z(), nxy, goff, gok, tid);
        load_psi_plane<TS>(rring[1], rsrc, z0, nz, g.wall_z(), nxy, goff, gok, tid);
    }
    const int lc = (ty + 1) * TS::RX + tx + 1;   // this cell's position in a ring plane
    for (int z = z0, j = 0; z < zend; ++z, ++j) {
        if (PSI_PF) {
            if (MULTIPHASE) {
                put_psi_plane<TS>(ring[(j + 2) & 3], pv, tid);
                if (z + 1 < zend) fetch_psi_plane<TS>(pv, psi, z + 2, nz, g.wall_z(), nxy, goff, gok, tid);
            }
            if (F16) {
                put_psi_plane<TS>(rring[(j + 2) & 3], rv, tid);
                if (z + 1 < zend) fetch_psi_plane<TS>(rv, rsrc, z + 2, nz, g.wall_z(), nxy, goff, gok, tid);
            }
        } else {
            if (MULTIPHASE) load_psi_plane<TS>(ring[(j + 2) & 3], psi, z + 1, nz, g.wall_z(), nxy, goff, gok, tid);
            if (F16) load_psi_plane<TS>(rring[(j + 2) & 3], rsrc, z + 1, nz, g.wall_z(), nxy, goff, gok, tid);
        }
        if (MULTIPHASE || F16) __syncthreads();
        if (!act_xy) continue;
#if LBM_ZM_PREFETCH
        float p[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) p[i] = pn[i];
        const uint32_t bits = bits_n;
        if (z + 1 < zend) {
            set_plane(o, z + 1, nz, nxy);
            bits_n = SOLIDS ? solid_bits32<Q>(g, nbmask, o.c, x, y, z + 1) : 0u;
            if (!(bits_n & 1u)) gather32<Q, PARITY, SOLIDS>(addr, o, bits_n, pn);
        }
        set_plane(o, z, nz, nxy);
        if (bits & 1u) continue;
#else
        set_plane(o, z, nz, nxy);
        const uint32_t bits = SOLIDS ? solid_bits32<Q>(g, nbmask, o.c, x, y, z) : 0u;
        if (bits & 1u) continue;
        float p[Q];
        gather32<Q, PARITY, SOLIDS>(addr, o, bits, p);
#endif
        if (F16) denorm<Q, SOLIDS>(p, bits, RsRing{&rring[j & 3][lc], &rring[(j + 1) & 3][lc],
                                                    &rring[(j + 2) & 3][lc], TS::RX});
        Forces Fo;
        if (MULTIPHASE) {
            Fo = stencil_forces3<Q, SOLIDS>(kp, &ring[j & 3][lc], &ring[(j + 1) & 3][lc], &ring[(j + 2) & 3][lc],
                                            TS::RX, bits);
        } else {
            Fo.fx = Fo.fy = Fo.fz = 0.f;
            Fo.qxx = Fo.qyy = Fo.qzz = Fo.qxy = Fo.qxz = Fo.qyz = 0.f;
            Fo.s2 = 0.f;
        }
        float rho, ux, uy, uz;
        collide<Q>(kp, p, Fo, rho, ux, uy, uz);
        if (!(rho > 0.0f) || !(fabsf(ux) + fabsf(uy) + fabsf(uz) < 1e30f)) atomicOr(status, ST_UNSTABLE);
        if (F16) normalize<Q>(p, __ldg(rown + o.c));
        store32<Q, PARITY, SOLIDS>(addr, o, bits, p);
    }
}

template <int PARITY, bool SOLIDS, bool MULTIPHASE, bool F16>
__global__ void __launch_bounds__(ZmTile::NT, ZM_MINB) collide_kernel(const KParams kp, const float* __restrict__ psi,
                                                                const uint32_t* __restrict__ nbmask,
                                                                unsigned* status, int zchunk,
                                                                const float* __restrict__ rsrc,
                                                                const float* __restrict__ rown) {
    __shared__ float ring[F16 ? 8 : 4][ZmTile::RP];
    const KGeom g{kp};
    const PlanePtrsT<typename std::conditional<F16, __half, float>::type> addr{kp};
    collide_tile<ZmTile, PARITY, SOLIDS, MULTIPHASE, F16, true>(kp, g, addr, psi, nbmask, status, blockIdx.x * ZM_BX,
                                                        blockIdx.y * ZM_BY, kp.zlo + (int)blockIdx.z * zchunk,
                                                        zchunk, kp.zhi, ring, ring + 4, rsrc, rown);
}

// ---- shifted FP16 store in the x-paired layout (KParams::paired: even nx, x periodic, no solid
// mask).  One thread per word, i.e. per cell pair (w, y, z) and (w + hx, y, z); every population
// slot is read and written as one half2 word, and the two cells share the address arithmetic.  A
// shift by one cell in x moves a word to the neighbouring word, with its two halves exchanged
// where the shift wraps around the row (w = 0 to the left, w = hx - 1 to the right).  Per cell
// the arithmetic and its order are those of the one-cell kernels above, so both layouts give the
// same populations bit for bit.

// word offsets of a pair's neighbourhood within a population plane (ncell / 2 words)
struct WOff {
    uint32_t c;
    uint32_t wo[3];   // words w-1, w, w+1 wrapped in [0, hx)
    uint32_t yo[3];   // rows y-1, y, y+1 wrapped, times hx
    uint32_t zo[3];   // planes z-1, z, z+1 wrapped, times ny hx
    __device__ __forceinline__ uint32_t nb(int dx, int dy, int dz) const { return zo[dz + 1] + yo[dy + 1] + wo[dx + 1]; }
};

__device__ __forceinline__ void set_wplane(WOff& o, int z, int nz, uint32_t wpl) {
    o.zo[0] = (uint32_t)wrap1(z - 1, nz) * wpl;
    o.zo[1] = (uint32_t)z * wpl;
    o.zo[2] = (uint32_t)wrap1(z + 1, nz) * wpl;
    o.c = o.zo[1] + o.yo[1] + o.wo[1];
}

struct WordPlanes {
    const KParams& kp;
    __device__ __forceinline__ uint32_t* ptr(int i, uint32_t off) const {
#if LBM_BOUNDS_CHECK
        if (i < 0 || i >= 27 || !kp.fq[i]) {
            atomicAdd(&lbm_bounds_count, 1ull);
            i = 0;
        }
#endif
        return reinterpret_cast<uint32_t*>(kp.fq[i]) + bounded(off, (unsigned long long)(kp.ncell / 2));
    }
};

constexpr uint32_t PERM_KEEP = 0x3210u, PERM_SWAP = 0x1032u;   // __byte_perm selectors: halves kept / exchanged

__device__ __forceinline__ float half_lo(uint32_t v) { return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu))); }
__device__ __forceinline__ float half_hi(uint32_t v) { return __half2float(__ushort_as_half((unsigned short)(v >> 16))); }

// slot words of the paired FP16 store: read once and written once per step.  Measured at 256^3 (step
// ms, D3Q19 / D3Q27, two repetitions): plain loads and stores 0.6453 / 0.8782; loads with a 256-byte L2
// prefetch 0.6420 / 0.8748; evict-first stores 0.6406 / 0.8777; both 0.6375 / 0.8745 (kept).
#ifndef LBM_LDWORD_HINT
#define LBM_LDWORD_HINT 2
#endif
#ifndef LBM_STWORD_CS
#define LBM_STWORD_CS 1
#endif
__device__ __forceinline__ uint32_t ldword(const uint32_t* p) {
#if LBM_LDWORD_HINT == 2
    uint32_t v;
    asm("ld.global.nc.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#else
    return __ldg(p);
#endif
}
__device__ __forceinline__ void stword(uint32_t* p, uint32_t v) {
#if LBM_STWORD_CS
    __stcs(p, v);
#else
    *p = v;
#endif
}

// AA gather of a pair's slot words (the paired counterpart of gather32); selL / selR exchange the
// halves of words fetched across the left / right end of the row
template <int PARITY, bool SOLIDS>
__device__ __forceinline__ void gather_pair(const WordPlanes& a, const WOff& o, uint32_t bits, uint32_t selL,
                                            uint32_t selR, uint32_t (&w)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (PARITY == 0 || i == 0 || (SOLIDS && ((bits >> OPP(i)) & 1u))) {
            w[i] = ldword(a.ptr(i, o.c));
        } else {
            const uint32_t v = ldword(a.ptr(OPP(i), o.nb(-EX(i), -EY(i), -EZ(i))));
            w[i] = EX(i) > 0 ? __byte_perm(v, 0u, selL) : (EX(i) < 0 ? __byte_perm(v, 0u, selR) : v);
        }
    }
}

// ... and the AA store of its post-collision words (the counterpart of store32)
template <int PARITY, bool SOLIDS>
__device__ __forceinline__ void store_pair(const WordPlanes& a, const WOff& o, uint32_t bits, uint32_t selL,
                                           uint32_t selR, const uint32_t (&w)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (PARITY == 0 || i == 0 || (SOLIDS && ((bits >> i) & 1u))) {
            stword(a.ptr(OPP(i), o.c), w[i]);
        } else {
            const uint32_t v = EX(i) > 0 ? __byte_perm(w[i], 0u, selR) : (EX(i) < 0 ? __byte_perm(w[i], 0u, selL) : w[i]);
            stword(a.ptr(i, o.nb(EX(i), EY(i), EZ(i))), v);
        }
    }
}

__device__ __forceinline__ void pair_offsets(WOff& o, int w, int y, int hx, int ny) {
    o.wo[0] = (uint32_t)wrap1(w - 1, hx);
    o.wo[1] = (uint32_t)w;
    o.wo[2] = (uint32_t)wrap1(w + 1, hx);
    o.yo[0] = (uint32_t)wrap1(y - 1, ny) * (uint32_t)hx;
    o.yo[1] = (uint32_t)y * (uint32_t)hx;
    o.yo[2] = (uint32_t)wrap1(y + 1, ny) * (uint32_t)hx;
}

// collide-stream pass over pairs: tiles of 32 pairs x PR_BY rows (64 x PR_BY cells) marching
// through a z-chunk, as collide_tile does for single cells.  The psi and writer-density rings
// hold, per pair position, the value at the low cell's neighbour and the one at the high cell's
// neighbour (exchanged where the position wraps around the row), in two planes, so that a warp
// reading one cell's stencil reads consecutive words (no bank conflicts).
constexpr int PR_BX = 32, PR_BY = 4, PR_NT = PR_BX * PR_BY;
// Resident blocks per SM and the next-plane word prefetch, measured at 256^3 (collide ms, D3Q19 /
// D3Q27): 4 / 3 blocks with prefetch 0.485 / 0.734 (no spills); 5 / 4 with prefetch 0.461 / 0.603
// (a few spilled registers); 6 / 5 with prefetch 0.456 / 0.695; 6 / 5 without 0.452 / 0.651; D3Q19
// without: 5 blocks 0.454, 7 blocks 0.444 (spilling up to 320 bytes).
// Kept: D3Q19 7 blocks without the prefetch, D3Q27 4 blocks with it.
#ifndef LBM_PR_MINB19
#define LBM_PR_MINB19 7
#endif
#ifndef LBM_PR_MINB27
#define LBM_PR_MINB27 4
#endif
#ifndef LBM_PR_PREFETCH
#define LBM_PR_PREFETCH (LBM_Q == 19 ? 0 : 1)
#endif
constexpr int PR_MINB = LBM_Q == 19 ? LBM_PR_MINB19 : LBM_PR_MINB27;
constexpr int PR_RX = PR_BX + 2, PR_RY = PR_BY + 2, PR_RP = PR_RX * PR_RY;
constexpr int PR_SLOTS = (PR_RP + PR_NT - 1) / PR_NT;

// where this thread's ring entries come from: natural offset of the low cell within a plane,
// whether the position lies in the domain, and whether its halves are exchanged
struct PairRingSrc {
    uint32_t off[PR_SLOTS];
    bool ok[PR_SLOTS], sw[PR_SLOTS];
};

__device__ __forceinline__ void fetch_pair_plane(float2 (&v)[PR_SLOTS], const float* __restrict__ fld, int zz, int nz,
                                                 int wall_z, uint32_t nxy, int hx, const PairRingSrc& g, int tid) {
    bool zok = true;
    if (zz < 0) { zok = !wall_z; zz += nz; } else if (zz >= nz) { zok = !wall_z; zz -= nz; }
    const uint32_t zb = (uint32_t)zz * nxy;
#pragma unroll
    for (int s = 0; s < PR_SLOTS; ++s) {
        const int k = tid + s * PR_NT;
        if (k < PR_RP && zok && g.ok[s]) {
            const float a = __ldg(fld + bounded(zb + g.off[s], (unsigned long long)nxy * nz));
            const float b = __ldg(fld + bounded(zb + g.off[s] + hx, (unsigned long long)nxy * nz));
            v[s] = g.sw[s] ? make_float2(b, a) : make_float2(a, b);
        } else {
            v[s] = make_float2(0.0f, 0.0f);
        }
    }
}
// a ring plane keeps the two halves apart (low cells' values, then high cells'), so that a warp
// reading one cell's stencil touches consecutive words
__device__ __forceinline__ void put_pair_plane(float (*slot)[PR_RP], const float2 (&v)[PR_SLOTS], int tid) {
#pragma unroll
    for (int s = 0; s < PR_SLOTS; ++s) {
        const int k = tid + s * PR_NT;
        if (k < PR_RP) {
            slot[0][k] = v[s].x;
            slot[1][k] = v[s].y;
        }
    }
}

// where a thread's ring entries come from (as collide_pair_kernel computes them)
__device__ __forceinline__ PairRingSrc pair_ring_src(int w0, int y0, int hx, int nx, int ny, int wall_y, int tid) {
    PairRingSrc src;
#pragma unroll
    for (int s = 0; s < PR_SLOTS; ++s) {
        const int k = tid + s * PR_NT;
        int pw = w0 - 1 + k % PR_RX, gy = y0 - 1 + k / PR_RX;
        bool ok = k < PR_RP, sw = false;
        if (pw < 0) { pw += hx; sw = true; } else if (pw >= hx) { pw -= hx; sw = true; }
        if (gy < 0) { ok &= !wall_y; gy += ny; } else if (gy >= ny) { ok &= !wall_y; gy -= ny; }
        // one wrap suffices for every position an active thread reads; anything still outside is unused
        ok = ok && pw >= 0 && pw < hx && gy >= 0 && gy < ny;
        src.ok[s] = ok;
        src.sw[s] = sw;
        src.off[s] = ok ? (uint32_t)gy * (uint32_t)nx + (uint32_t)pw : 0u;
    }
    return src;
}

// density + psi pass over pairs: the counterpart of psi_kernel for the paired layout, one plane per
// block.  (A z-marching variant with the writers' densities in a shared ring, read at fixed offsets,
// measured slower: 0.242 against 0.199 ms at 256^3 D3Q19; the per-population reads hit L1.)
template <int PARITY, bool SOLIDS>
__global__ void __launch_bounds__(PSI_BX * PSI_BY) psi_pair_kernel(KParams kp, float* __restrict__ psi,
                                                                 unsigned* status, const float* __restrict__ rsrc,
                                                                 float* __restrict__ rdst) {
    const int hx = kp.hx, nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int w = blockIdx.x * PSI_BX + threadIdx.x, y = blockIdx.y * PSI_BY + threadIdx.y, z = blockIdx.z;
    if (w >= hx || y >= ny) return;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
    WOff o;
    pair_offsets(o, w, y, hx, ny);
    set_wplane(o, z, nz, (uint32_t)hx * (uint32_t)ny);
    const uint32_t selL = w == 0 ? PERM_SWAP : PERM_KEEP, selR = w == hx - 1 ? PERM_SWAP : PERM_KEEP;
    const uint32_t bits = SOLIDS ? solid_bits32<Q>(KGeom{kp}, nullptr, 0u, w, y, z) : 0u;
    uint32_t wv[Q];
    gather_pair<PARITY, SOLIDS>(WordPlanes{kp}, o, bits, selL, selR, wv);
    // natural neighbourhoods of the two cells, for the writers' densities
    Off32 on[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int x = w + h * hx;
        on[h].xo[0] = (uint32_t)wrap1(x - 1, nx);
        on[h].xo[1] = (uint32_t)x;
        on[h].xo[2] = (uint32_t)wrap1(x + 1, nx);
        on[h].yo[0] = (uint32_t)wrap1(y - 1, ny) * (uint32_t)nx;
        on[h].yo[1] = (uint32_t)y * (uint32_t)nx;
        on[h].yo[2] = (uint32_t)wrap1(y + 1, ny) * (uint32_t)nx;
        set_plane(on[h], z, nz, nxy);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float p[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) p[i] = h ? half_hi(wv[i]) : half_lo(wv[i]);
        denorm<Q, SOLIDS>(p, bits, RsOff32{rsrc, on[h]});
        float rho = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) rho += p[i];
        rdst[on[h].c] = rho;
        if (kp.multiphase) psi[bounded(on[h].c, (unsigned long long)nxy * nz)] = eval_psi(kp, rho, status);
    }
}

template <int PARITY, bool SOLIDS, bool MULTIPHASE>
__global__ void __launch_bounds__(PR_NT, PR_MINB) collide_pair_kernel(const KParams kp, const float* __restrict__ psi,
                                                                     unsigned* status, int zchunk,
                                                                     const float* __restrict__ rsrc,
                                                                     const float* __restrict__ rown) {
    __shared__ float ring[4][2][PR_RP];    // psi (low cells, high cells)
    __shared__ float rring[4][2][PR_RP];   // densities the slots were written with
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + PR_BX * ty;
    const int hx = kp.hx, nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int w0 = blockIdx.x * PR_BX, y0 = blockIdx.y * PR_BY;
    const int w = w0 + tx, y = y0 + ty;
    const bool act = w < hx && y < ny;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny, wpl = (uint32_t)hx * (uint32_t)ny;
    const int z0 = kp.zlo + (int)blockIdx.z * zchunk;
    const int zend = min(z0 + zchunk, kp.zhi);
    const KGeom g{kp};
    const WordPlanes addr{kp};

    const PairRingSrc src = pair_ring_src(w0, y0, hx, nx, ny, g.wall_y(), tid);
    WOff o;
    pair_offsets(o, w < hx ? w : 0, y < ny ? y : 0, hx, ny);
    const uint32_t selL = w == 0 ? PERM_SWAP : PERM_KEEP, selR = w == hx - 1 ? PERM_SWAP : PERM_KEEP;
    const uint32_t rowA = (uint32_t)(y < ny ? y : 0) * (uint32_t)nx + (uint32_t)(w < hx ? w : 0);   // low cell in its plane

    // words and own densities of the first plane, then of plane z+1 while plane z is computed
    uint32_t wn[Q];
    float rn[2] = {0.0f, 0.0f};
    uint32_t bits_n = 0u;
    if (act) {
        set_wplane(o, z0, nz, wpl);
        bits_n = SOLIDS ? solid_bits32<Q>(g, nullptr, 0u, w, y, z0) : 0u;
        gather_pair<PARITY, SOLIDS>(addr, o, bits_n, selL, selR, wn);
        rn[0] = __ldg(rown + (uint32_t)z0 * nxy + rowA);
        rn[1] = __ldg(rown + (uint32_t)z0 * nxy + rowA + hx);
    }
    float2 pv[PR_SLOTS], rv[PR_SLOTS];
    if (MULTIPHASE) fetch_pair_plane(pv, psi, z0 + 1, nz, g.wall_z(), nxy, hx, src, tid);
    fetch_pair_plane(rv, rsrc, z0 + 1, nz, g.wall_z(), nxy, hx, src, tid);
    {
        float2 t0[PR_SLOTS], t1[PR_SLOTS];
        if (MULTIPHASE) {
            fetch_pair_plane(t0, psi, z0 - 1, nz, g.wall_z(), nxy, hx, src, tid);
            fetch_pair_plane(t1, psi, z0, nz, g.wall_z(), nxy, hx, src, tid);
            put_pair_plane(ring[0], t0, tid);
            put_pair_plane(ring[1], t1, tid);
        }
        fetch_pair_plane(t0, rsrc, z0 - 1, nz, g.wall_z(), nxy, hx, src, tid);
        fetch_pair_plane(t1, rsrc, z0, nz, g.wall_z(), nxy, hx, src, tid);
        put_pair_plane(rring[0], t0, tid);
        put_pair_plane(rring[1], t1, tid);
    }
    const int lc = (ty + 1) * PR_RX + tx + 1;   // this pair's position in a ring plane
    for (int z = z0, j = 0; z < zend; ++z, ++j) {
        if (MULTIPHASE) {
            put_pair_plane(ring[(j + 2) & 3], pv, tid);
            if (z + 1 < zend) fetch_pair_plane(pv, psi, z + 2, nz, g.wall_z(), nxy, hx, src, tid);
        }
        put_pair_plane(rring[(j + 2) & 3], rv, tid);
        if (z + 1 < zend) fetch_pair_plane(rv, rsrc, z + 2, nz, g.wall_z(), nxy, hx, src, tid);
        __syncthreads();
        if (!act) continue;
        uint32_t wv[Q];
        if (!LBM_PR_PREFETCH && z > z0) {   // no prefetch: this plane's words now
            set_wplane(o, z, nz, wpl);
            bits_n = SOLIDS ? solid_bits32<Q>(g, nullptr, 0u, w, y, z) : 0u;
            gather_pair<PARITY, SOLIDS>(addr, o, bits_n, selL, selR, wn);
            rn[0] = __ldg(rown + (uint32_t)z * nxy + rowA);
            rn[1] = __ldg(rown + (uint32_t)z * nxy + rowA + hx);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) wv[i] = wn[i];
        const float rown_c[2] = {rn[0], rn[1]};
        const uint32_t bits = bits_n;
        if (LBM_PR_PREFETCH && z + 1 < zend) {
            set_wplane(o, z + 1, nz, wpl);
            bits_n = SOLIDS ? solid_bits32<Q>(g, nullptr, 0u, w, y, z + 1) : 0u;
            gather_pair<PARITY, SOLIDS>(addr, o, bits_n, selL, selR, wn);
            rn[0] = __ldg(rown + (uint32_t)(z + 1) * nxy + rowA);
            rn[1] = __ldg(rown + (uint32_t)(z + 1) * nxy + rowA + hx);
        }
        set_wplane(o, z, nz, wpl);
        // wv ends up holding the outputs: the low cell's packed results replace the low halves it
        // has consumed, then the high cell's replace the high halves (no second array of words)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float p[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) p[i] = h ? half_hi(wv[i]) : half_lo(wv[i]);
            denorm<Q, SOLIDS>(p, bits, RsRing{&rring[j & 3][h][lc], &rring[(j + 1) & 3][h][lc],
                                              &rring[(j + 2) & 3][h][lc], PR_RX});
            Forces Fo;
            if (MULTIPHASE) {
                Fo = stencil_forces3<Q, SOLIDS>(kp, &ring[j & 3][h][lc], &ring[(j + 1) & 3][h][lc],
                                                &ring[(j + 2) & 3][h][lc], PR_RX, bits);
            } else {
                Fo.fx = Fo.fy = Fo.fz = 0.f;
                Fo.qxx = Fo.qyy = Fo.qzz = Fo.qxy = Fo.qxz = Fo.qyz = 0.f;
                Fo.s2 = 0.f;
            }
            float rho, ux, uy, uz;
            collide<Q>(kp, p, Fo, rho, ux, uy, uz);
            if (!(rho > 0.0f) || !(fabsf(ux) + fabsf(uy) + fabsf(uz) < 1e30f)) atomicOr(status, ST_UNSTABLE);
            normalize<Q>(p, rown_c[h]);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const uint32_t hv = (uint32_t)__half_as_ushort(__float2half_rn(p[i]));
                wv[i] = h ? ((wv[i] & 0x0000ffffu) | (hv << 16)) : ((wv[i] & 0xffff0000u) | hv);
            }
        }
        store_pair<PARITY, SOLIDS>(addr, o, bits, selL, selR, wv);
    }
}

// ---- one-pass update with two population copies (periodic domains without solids, FP32).
// kp.fq holds the copy being read (pull layout: population i of x is slot i of x - e_i, written by
// x - e_i in the previous step), kp.gq the copy this step writes (slot i of x = f*_i(x)).  Nothing
// writes kp.fq during the launch, so a block can pull the populations of cells it does not own:
// it computes rho and psi of its tile and of a one-cell halo itself, one plane ahead of the
// collision, with the same summation order and EOS code as the density/psi pass.  The step reads
// and writes each population once and needs no psi field.
__device__ __forceinline__ void pull_offsets(Off32& o, int x, int y, int nx, int ny) {
    o.xo[0] = (uint32_t)wrap1(x - 1, nx);
    o.xo[1] = (uint32_t)x;
    o.xo[2] = (uint32_t)wrap1(x + 1, nx);
    o.yo[0] = (uint32_t)wrap1(y - 1, ny) * (uint32_t)nx;
    o.yo[1] = (uint32_t)y * (uint32_t)nx;
    o.yo[2] = (uint32_t)wrap1(y + 1, ny) * (uint32_t)nx;
}

// Tiles of 32 x BY cells; the ring plane is (32 + 2) x (BY + 2) with a border of 2 (32 + 2) + 2 BY
// cells, whose densities the first threads of the block compute besides their own.
template <bool MULTIPHASE, int BY, int MINB>
__global__ void __launch_bounds__(32 * BY, MINB) collide_onepass_kernel(const KParams kp, unsigned* status,
                                                                        int zchunk) {
    constexpr int RX = 34, RY = BY + 2, RP = RX * RY, HALO = 2 * RX + 2 * BY;
    static_assert(HALO <= 32 * BY, "one border cell per thread at most");
    __shared__ float ring[4][RP];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * BY, z0 = blockIdx.z * zchunk;
    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
    const int zend = min(z0 + zchunk, nz);
    const PlanePtrs rd{kp};

    // this thread's ring cell (its own cell, wrapped where the tile overhangs the domain)
    Off32 o;
    pull_offsets(o, x % nx, y % ny, nx, ny);
    const int lc = (ty + 1) * RX + tx + 1;
    // and one border cell of the ring plane for HALO threads, spread evenly over the warps (the
    // first lanes of each), so that every warp reaches the plane's barrier with the same work
    constexpr int NWARP = BY, PER_WARP = (HALO + NWARP - 1) / NWARP;
    static_assert(PER_WARP <= 32, "one border cell per lane at most");
    const int hb = (tid & 31) < PER_WARP ? (tid >> 5) * PER_WARP + (tid & 31) : HALO;   // border index
    const bool has_halo = hb < HALO;
    Off32 oh;
    int hl = 0;
    if (MULTIPHASE && has_halo) {
        int rx, ry;
        if (hb < RX) { rx = hb; ry = 0; }
        else if (hb < 2 * RX) { rx = hb - RX; ry = RY - 1; }
        else if (hb < 2 * RX + BY) { rx = 0; ry = 1 + hb - 2 * RX; }
        else { rx = RX - 1; ry = 1 + hb - 2 * RX - BY; }
        hl = ry * RX + rx;
        pull_offsets(oh, (x0 - 1 + rx + nx) % nx, (y0 - 1 + ry + ny) % ny, nx, ny);
    }

    // psi of plane zz at this thread's ring cells; the own cell's populations are returned in p
    auto plane_psi = [&](float* slot, int zz, float (&p)[Q]) {
        zz = wrap1(zz, nz);
        set_plane(o, zz, nz, nxy);
        gather32<Q, 2, false>(rd, o, 0u, p);
        if (MULTIPHASE) {
            float rho = 0.0f;
#pragma unroll
            for (int i = 0; i < Q; ++i) rho += p[i];
            slot[lc] = eval_psi(kp, rho, status);
            if (has_halo) {
                set_plane(oh, zz, nz, nxy);
                float q[Q];
                gather32<Q, 2, false>(rd, oh, 0u, q);
                float rh = 0.0f;
#pragma unroll
                for (int i = 0; i < Q; ++i) rh += q[i];
                slot[hl] = eval_psi(kp, rh, status);
            }
        }
    };

    float pn[Q];
    if (MULTIPHASE) {
        float tmp[Q];
        plane_psi(ring[0], z0 - 1, tmp);
    }
    plane_psi(ring[1], z0, pn);
    for (int z = z0, j = 0; z < zend; ++z, ++j) {
        float p[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) p[i] = pn[i];
        if (MULTIPHASE || z + 1 < zend) plane_psi(ring[(j + 2) & 3], z + 1, pn);
        if (MULTIPHASE) __syncthreads();
        if (!act) continue;
        set_plane(o, z, nz, nxy);
        Forces Fo;
        if (MULTIPHASE) {
            Fo = stencil_forces3<Q, false>(kp, &ring[j & 3][lc], &ring[(j + 1) & 3][lc], &ring[(j + 2) & 3][lc],
                                           RX, 0u);
        } else {
            Fo.fx = Fo.fy = Fo.fz = 0.f;
            Fo.qxx = Fo.qyy = Fo.qzz = Fo.qxy = Fo.qxz = Fo.qyz = 0.f;
            Fo.s2 = 0.f;
        }
        float rho, ux, uy, uz;
        collide<Q>(kp, p, Fo, rho, ux, uy, uz);
        if (!(rho > 0.0f) || !(fabsf(ux) + fabsf(uy) + fabsf(uz) < 1e30f)) atomicOr(status, ST_UNSTABLE);
#pragma unroll
        for (int i = 0; i < Q; ++i) kp.gq[i][bounded(o.c, (unsigned long long)kp.ncell)] = p[i];
    }
}

// ---- one-pass step with the pulled populations staged by TMA (full 32 x 4 tiles: nx a multiple of
// 32, ny of 4).  For every plane c a block needs, one tensor copy per population i brings the slots of
// storage plane c - e_iz for x0 - 4 .. x0 + 35 and y0 - 2 .. y0 + 5 (a 40 x 8 box; starting at x0 - 4
// keeps every copy on a 16-byte boundary) into shared memory, where the block's cells and its one-cell
// border read their pulled populations (population i of cell x is slot i of x - e_i).  Two box sets
// alternate: the copies for plane c + 2 are issued as soon as plane c has been consumed, so they land
// while plane c - 1 is collided and no thread waits on a load of its own.  Box positions outside the
// domain come back as zeros; the tiles at the x and y faces fill their periodic images from global
// memory.  The arithmetic and its order are those of collide_onepass_kernel, so the results are the
// same bit for bit.  Every wait on a copy is bounded in time: past `wait_cycles` the whole block
// raises ST_TIMEOUT, waits (bounded again) for its copies still in flight and returns.
constexpr int OT_HX = 40, OT_HY = 8, OT_BOX = OT_HX * OT_HY;
constexpr int OT_RX = 34, OT_RY = 6, OT_RP = OT_RX * OT_RY, OT_HALO = 2 * OT_RX + 2 * 4;
constexpr int OT_MINB = LBM_Q == 19 ? 4 : 3;

struct OtShared {
    float pop[2][Q][OT_BOX];     // two box sets, one box per population
    float ring[4][OT_RP];        // psi of planes z-1, z, z+1 (and the next)
    unsigned long long bar[2];   // completion of each box set's copies
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// one thread: the copies of plane c into box set b, completing on bar[b] (extra: bytes expected
// beyond those the copies deliver -- nonzero only to exercise the timeout path)
__device__ __forceinline__ void ot_issue(OtShared& sm, int b, const CUtensorMap* map, int x0, int y0, int c, int nz,
                                         unsigned extra) {
    const uint32_t bar = smem_u32(&sm.bar[b]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"((unsigned)(Q * OT_BOX * sizeof(float)) + extra) : "memory");
    const int cw = wrap1(c, nz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int pz = wrap1(cw - EZ(i), nz);
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
            :: "r"(smem_u32(&sm.pop[b][i][0])), "l"(reinterpret_cast<uint64_t>(map)), "r"(x0 - 4), "r"(y0 - 2), "r"(pz),
               "r"(i), "r"(bar)
            : "memory");
    }
}

// bounded wait for phase `ph` of bar[b]; false once wait_cycles have passed
__device__ __forceinline__ bool ot_wait(OtShared& sm, int b, unsigned ph, long long wait_cycles) {
    const uint32_t bar = smem_u32(&sm.bar[b]);
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok) : "r"(bar), "r"(ph) : "memory");
        if (ok) return true;
        if (clock64() - t0 > wait_cycles) return false;
    }
}

// Plane c from box set b: wait for its copies (bounded), fill the periodic images at the faces, then psi
// of the tile and of its border into `slot`; the own cell's pulled populations into p.  False if the
// wait ran out on any thread of the block (the decision is block-wide).
template <bool MULTIPHASE>
__device__ __forceinline__ bool ot_stage(const KParams& kp, OtShared& sm, int c, int b, float* slot, float (&p)[Q],
                                         unsigned& phase, unsigned& pending, long long wait_cycles, unsigned* status,
                                         int tid, int x0, int y0, bool face, int lc, bool has_halo, int rx, int ry,
                                         int hl) {
    const int tx = tid & 31, ty = tid >> 5;
    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
    const bool ok = ot_wait(sm, b, (phase >> b) & 1u, wait_cycles);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1u << b;
    pending &= ~(1u << b);
    if (face) {
        // positions outside [0, nx) x [0, ny) among the needed x0-2 .. x0+33, y0-2 .. y0+5
        const int nL = x0 == 0, nR = x0 + 32 == nx, nT = y0 == 0, nB = y0 + 4 == ny;
        const int per = 16 * nL + 16 * nR + 72 * nT + 72 * nB;
        const int cw = wrap1(c, nz);
        for (int k = tid; k < Q * per; k += 128) {
            const int i = k % Q;
            int r = k / Q, lx, ly;
            if (nL && r < 16) { lx = 2 + (r & 1); ly = r >> 1; }
            else {
                r -= 16 * nL;
                if (nR && r < 16) { lx = 36 + (r & 1); ly = r >> 1; }
                else {
                    r -= 16 * nR;
                    if (nT && r < 72) { lx = 2 + r % 36; ly = r / 36; }
                    else { r -= 72 * nT; lx = 2 + r % 36; ly = 6 + r / 36; }
                }
            }
            int gx = x0 - 4 + lx, gy = y0 - 2 + ly;
            gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
            gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
            // population i's plane base and storage plane c - e_iz, selected with compile-time indices
            const float* src = kp.fq[0];
            int pz = cw;
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (q == i) {
                    src = kp.fq[q];
                    pz = wrap1(cw - EZ(q), nz);
                }
            sm.pop[b][i][ly * OT_HX + lx] =
                __ldg(src + bounded((uint32_t)pz * nxy + (uint32_t)gy * (uint32_t)nx + (uint32_t)gx,
                                    (unsigned long long)kp.ncell));
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) p[i] = sm.pop[b][i][(ty + 2 - EY(i)) * OT_HX + (tx + 4 - EX(i))];
    if (MULTIPHASE) {
        float rho = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) rho += p[i];
        slot[lc] = eval_psi(kp, rho, status);
        if (has_halo) {
            float rh = 0.0f;
#pragma unroll
            for (int i = 0; i < Q; ++i) rh += sm.pop[b][i][(ry + 1 - EY(i)) * OT_HX + (rx + 3 - EX(i))];
            slot[hl] = eval_psi(kp, rh, status);
        }
    }
    __syncthreads();   // the box set has been read; psi of plane c is in the ring
    return true;
}

// after a wait ran out: raise ST_TIMEOUT and wait (bounded again) for the copies still in flight
__device__ __forceinline__ void ot_bail(OtShared& sm, unsigned phase, unsigned pending, long long wait_cycles,
                                        unsigned* status, int tid) {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    for (int b = 0; b < 2; ++b)
        if ((pending >> b) & 1u) (void)ot_wait(sm, b, (phase >> b) & 1u, wait_cycles);
}

template <bool MULTIPHASE>
__global__ void __launch_bounds__(128, OT_MINB) collide_onepass_tma_kernel(const KParams kp,
                                                                          const __grid_constant__ CUtensorMap map,
                                                                          unsigned* status, int zchunk,
                                                                          unsigned extra_tx, long long wait_cycles) {
    extern __shared__ __align__(128) unsigned char ot_raw[];
    OtShared& sm = *reinterpret_cast<OtShared*>(ot_raw);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 4, z0 = blockIdx.z * zchunk;
    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
    const int zend = min(z0 + zchunk, nz);
    const int base = z0 - 1;                        // first plane staged (psi only)
    const bool face = x0 == 0 || x0 + 32 == nx || y0 == 0 || y0 + 4 == ny;
    const int lc = (ty + 1) * OT_RX + tx + 1;
    const uint32_t own = (uint32_t)(y0 + ty) * (uint32_t)nx + (uint32_t)(x0 + tx);
    // one border cell of the ring plane for 19 lanes of each warp (as collide_onepass_kernel)
    constexpr int PER_WARP = (OT_HALO + 3) / 4;
    const int hb = (tid & 31) < PER_WARP ? (tid >> 5) * PER_WARP + (tid & 31) : OT_HALO;
    const bool has_halo = MULTIPHASE && hb < OT_HALO;
    int rx = 0, ry = 0;
    if (has_halo) {
        if (hb < OT_RX) { rx = hb; ry = 0; }
        else if (hb < 2 * OT_RX) { rx = hb - OT_RX; ry = OT_RY - 1; }
        else if (hb < 2 * OT_RX + 4) { rx = 0; ry = 1 + hb - 2 * OT_RX; }
        else { rx = OT_RX - 1; ry = 1 + hb - 2 * OT_RX - 4; }
    }
    const int hl = ry * OT_RX + rx;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&sm.bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&sm.bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned phase = 0u;     // bit b: the completion phase box set b waits for next
    unsigned pending = 3u;   // bit b: box set b has copies in flight
    if (tid == 0) {
        ot_issue(sm, 0, &map, x0, y0, base, nz, extra_tx);
        ot_issue(sm, 1, &map, x0, y0, base + 1, nz, extra_tx);
    }

    float pn[Q];
    {
        float tmp[Q];
        if (!ot_stage<MULTIPHASE>(kp, sm, base, 0, sm.ring[0], tmp, phase, pending, wait_cycles, status, tid, x0, y0, face,
                                  lc, has_halo, rx, ry, hl))
            return ot_bail(sm, phase, pending, wait_cycles, status, tid);
    }
    if (tid == 0 && base + 2 <= zend) ot_issue(sm, 0, &map, x0, y0, base + 2, nz, extra_tx);
    if (base + 2 <= zend) pending |= 1u;
    if (!ot_stage<MULTIPHASE>(kp, sm, z0, 1, sm.ring[1], pn, phase, pending, wait_cycles, status, tid, x0, y0, face, lc,
                              has_halo, rx, ry, hl))
        return ot_bail(sm, phase, pending, wait_cycles, status, tid);
    if (tid == 0 && base + 3 <= zend) ot_issue(sm, 1, &map, x0, y0, base + 3, nz, extra_tx);
    if (base + 3 <= zend) pending |= 2u;
    for (int z = z0, j = 0; z < zend; ++z, ++j) {
        float p[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) p[i] = pn[i];
        const int c = z + 1, b = (c - base) & 1;
        if (!ot_stage<MULTIPHASE>(kp, sm, c, b, sm.ring[(j + 2) & 3], pn, phase, pending, wait_cycles, status, tid, x0,
                                  y0, face, lc, has_halo, rx, ry, hl))
            return ot_bail(sm, phase, pending, wait_cycles, status, tid);
        if (tid == 0 && c + 2 <= zend) ot_issue(sm, b, &map, x0, y0, c + 2, nz, extra_tx);
        if (c + 2 <= zend) pending |= 1u << b;
        Forces Fo;
        if (MULTIPHASE) {
            Fo = stencil_forces3<Q, false>(kp, &sm.ring[j & 3][lc], &sm.ring[(j + 1) & 3][lc],
                                           &sm.ring[(j + 2) & 3][lc], OT_RX, 0u);
        } else {
            Fo.fx = Fo.fy = Fo.fz = 0.f;
            Fo.qxx = Fo.qyy = Fo.qzz = Fo.qxy = Fo.qxz = Fo.qyz = 0.f;
            Fo.s2 = 0.f;
        }
        float rho, ux, uy, uz;
        collide<Q>(kp, p, Fo, rho, ux, uy, uz);
        if (!(rho > 0.0f) || !(fabsf(ux) + fabsf(uy) + fabsf(uz) < 1e30f)) atomicOr(status, ST_UNSTABLE);
        const uint32_t cell = (uint32_t)z * nxy + own;
#pragma unroll
        for (int i = 0; i < Q; ++i) kp.gq[i][bounded(cell, (unsigned long long)kp.ncell)] = p[i];
    }
}

// natural-order populations (plane i at fin + i * fstride) -> one-pass layout (slot i of x - e_i)
__global__ void pull_store_kernel(KParams kp, const float* __restrict__ fin, long long fstride,
                                  float* __restrict__ fout) {
    const long long n = kp.ncell;
    const long long nxy = (long long)kp.nx * kp.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const Cell c = make_cell(kp, (int)(idx % kp.nx), (int)((idx / kp.nx) % kp.ny), (int)(idx / nxy));
#pragma unroll
        for (int i = 0; i < Q; ++i) fout[i * kp.plane + idx] = fin[i * fstride + c.nb(EX(i), EY(i), EZ(i))];
    }
}

// multi-domain collide-stream pass: one block per tile of any member of the launch's table;
// physics by value; tiles of shape S of BATCH_SHAPES
template <int PARITY, bool SOLIDS, bool MULTIPHASE, int S>
__global__ void __launch_bounds__(BatchTileShape<S>::NT, batch_minb<S>()) collide_batch_kernel(
        const KParams phys, const __grid_constant__ BatchDomTable tab, const BatchTile* __restrict__ tiles) {
    using TS = BatchTileShape<S>;
    using TN = TileShape<BATCH_NARROW_BX, TS::NT / BATCH_NARROW_BX>;   // narrow tiles at the ends of rows
    static_assert(TN::RP <= TS::RP, "a narrow tile's ring fits the block's");
    __shared__ float ring[4][TS::RP];
    const BatchTile t = tiles[blockIdx.x];
    const BatchDom& m = tab.d[t.d];
    const DGeom g{m};
    const DomPlanes addr{m};
    if (TS::BX != BATCH_NARROW_BX && t.narrow)
        collide_tile<TN, PARITY, SOLIDS, MULTIPHASE, false, !SOLIDS, DGeom, DomPlanes, true>(
            phys, g, addr, m.psi, m.nbmask, m.status, t.x0, t.y0, t.z0, t.zc, g.nz(),
            reinterpret_cast<float (*)[TN::RP]>(&ring[0][0]), nullptr, nullptr, nullptr);
    else
        collide_tile<TS, PARITY, SOLIDS, MULTIPHASE, false, !SOLIDS>(phys, g, addr, m.psi, m.nbmask, m.status, t.x0,
                                                                    t.y0, t.z0, t.zc, g.nz(), ring, nullptr, nullptr,
                                                                    nullptr);
}

// ---- initialisation: f_bar = M^-1 m^eq(rho, u) (Eq. e13), natural layout
// F16: slot i of x is written relative to the density of x - e_i (x itself where that neighbour
// is solid), the cell that writes it in the AA streaming; rdst receives the initial densities.
template <bool F16>
__global__ void init_kernel(KParams kp, void* __restrict__ fv, const float* __restrict__ rho_in,
                            const float* __restrict__ u_in, const uint32_t* __restrict__ nbmask,
                            float* __restrict__ rdst) {
    using T = typename std::conditional<F16, __half, float>::type;
    T* f = reinterpret_cast<T*>(fv);
    const long long n = kp.ncell;
    const long long nxy = (long long)kp.nx * kp.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        float out[Q];
        const bool solid = nbmask && (__ldg(nbmask + idx) & 1u);
        if (solid) {
#pragma unroll
            for (int i = 0; i < Q; ++i) out[i] = 0.0f;
        } else {
            const float rho = rho_in[idx];
            const float ux = u_in[idx], uy = u_in[n + idx], uz = u_in[2 * n + idx];
            const float cs2 = 1.0f / 3.0f, cs4 = 1.0f / 9.0f, cs6 = 1.0f / 27.0f;
            const float uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
            float m[Q];
            m[0] = rho;
            m[1] = rho * ux;
            m[2] = rho * uy;
            m[3] = rho * uz;
            m[4] = rho * ux * uy;
            m[5] = rho * ux * uz;
            m[6] = rho * uy * uz;
            m[7] = rho * (1.0f + uxx + uyy + uzz);
            m[8] = rho * (uxx - uyy);
            m[9] = rho * (uxx - uzz);
            m[10] = cs2 * rho * ux;
            m[11] = cs2 * rho * ux;
            m[12] = cs2 * rho * uy;
            m[13] = cs2 * rho * uz;
            m[14] = cs2 * rho * uy;
            m[15] = cs2 * rho * uz;
            if (Q == 27) m[MP<Q>(16)] = 0.0f;
            m[MP<Q>(17)] = cs2 * rho * (cs2 + uxx + uyy);
            m[MP<Q>(18)] = cs2 * rho * (cs2 + uxx + uzz);
            m[MP<Q>(19)] = cs2 * rho * (cs2 + uyy + uzz);
            if (Q == 27) {
                m[MP<Q>(20)] = cs2 * rho * uy * uz;
                m[MP<Q>(21)] = cs2 * rho * ux * uz;
                m[MP<Q>(22)] = cs2 * rho * ux * uy;
                m[MP<Q>(23)] = cs4 * rho * ux;
                m[MP<Q>(24)] = cs4 * rho * uy;
                m[MP<Q>(25)] = cs4 * rho * uz;
                m[MP<Q>(26)] = cs4 * rho * (uxx + uyy + uzz) + cs6 * rho;
            }
            to_pops<Q>(m, out);
            if (F16) {
                const Cell c = make_cell(kp, (int)(idx % kp.nx), (int)((idx / kp.nx) % kp.ny), (int)(idx / nxy));
                const uint32_t bits = solid_bits<Q>(kp, nbmask, c);
                const float* r = rho_in;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const bool own = i == 0 || ((bits >> OPP(i)) & 1u);
                    const float rw = own ? rho : __ldg(r + c.nb(-EX(i), -EY(i), -EZ(i)));
                    out[i] = out[i] / rw - OMEGA<Q>(i);
                }
            }
        }
        if (F16) rdst[idx] = solid ? 1.0f : rho_in[idx];
        long long pi = idx;
        if (F16 && kp.paired) {
            const int x = (int)(idx % kp.nx);
            pi = idx - x + pair_pos(x, kp.hx);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) stpop(f + i * kp.plane + pi, out[i]);
    }
}

// ---- shifted FP16 store from natural-order populations (checkpoint restore): densities, then
// the slot values relative to them
__global__ void f16_density_kernel(KParams kp, const float* __restrict__ fin, const uint32_t* __restrict__ nbmask,
                                   float* __restrict__ rdst) {
    const long long n = kp.ncell;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        float rho = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) rho += fin[i * n + idx];
        rdst[idx] = (nbmask && (__ldg(nbmask + idx) & 1u)) ? 1.0f : rho;
    }
}

__global__ void f16_pack_kernel(KParams kp, const float* __restrict__ fin, const uint32_t* __restrict__ nbmask,
                                const float* __restrict__ rsrc, __half* __restrict__ f) {
    const long long n = kp.ncell;
    const long long nxy = (long long)kp.nx * kp.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const Cell c = make_cell(kp, (int)(idx % kp.nx), (int)((idx / kp.nx) % kp.ny), (int)(idx / nxy));
        const uint32_t bits = solid_bits<Q>(kp, nbmask, c);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float h = 0.0f;
            if (!(bits & 1u)) {
                const bool own = i == 0 || ((bits >> OPP(i)) & 1u);
                const float rw = own ? __ldg(rsrc + idx) : __ldg(rsrc + c.nb(-EX(i), -EY(i), -EZ(i)));
                h = fin[i * n + idx] / rw - OMEGA<Q>(i);
            }
            f[i * kp.plane + c.pidx] = __float2half_rn(h);
        }
    }
}

// ---- macroscopic output: rho, u = (sum f e + F/2)/rho, FP64 block partial sums
template <int PARITY, bool SOLIDS, bool MULTIPHASE, bool F16>
__global__ void __launch_bounds__(CS_BX * CS_BY * CS_BZ) moments_kernel(KParams kp, const void* __restrict__ fv,
                                                                       const float* __restrict__ psi,
                                                                       const uint32_t* __restrict__ nbmask,
                                                                       float* __restrict__ rho_out,
                                                                       float* __restrict__ u_out,
                                                                       double* __restrict__ partials,
                                                                       const float* __restrict__ rsrc) {
    using T = typename std::conditional<F16, __half, float>::type;
    const T* f = reinterpret_cast<const T*>(fv);
    __shared__ PsiTile<CS_BX, CS_BY, CS_BZ> tile;
    __shared__ double red[4][CS_BX * CS_BY * CS_BZ / 32];
    const int x0 = blockIdx.x * CS_BX, y0 = blockIdx.y * CS_BY, z0 = blockIdx.z * CS_BZ;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    const int tid = threadIdx.x + CS_BX * (threadIdx.y + CS_BY * threadIdx.z);
    const bool inside = x < kp.nx && y < kp.ny && z < kp.nz;
    Cell c;
    uint32_t bits = 0u;
    float p[Q];
    bool active = false;
    if (inside) {
        c = make_cell(kp, x, y, z);
        bits = SOLIDS ? solid_bits<Q>(kp, nbmask, c) : 0u;
        active = !(bits & 1u);
        if (active) {
            gather<Q, PARITY, SOLIDS>(kp, f, c, bits, p);
            if (F16) denorm<Q, SOLIDS>(p, bits, RsCell{rsrc, c});
        }
    }
    if (MULTIPHASE) {
        tile.load(kp, psi, x0, y0, z0, tid);
        __syncthreads();
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (active) {
        Forces Fo;
        if (MULTIPHASE) {
            Fo = stencil_forces<Q, SOLIDS>(kp, tile.at(threadIdx.x, threadIdx.y, threadIdx.z),
                                           PsiTile<CS_BX, CS_BY, CS_BZ>::TX,
                                           PsiTile<CS_BX, CS_BY, CS_BZ>::TX * PsiTile<CS_BX, CS_BY, CS_BZ>::TY, bits);
        } else {
            Fo.fx = Fo.fy = Fo.fz = 0.f;
        }
        float m[Q];
        to_moments<Q>(p, m);
        const float rho = m[0];
        const float jx = m[1] + 0.5f * (Fo.fx + rho * kp.gx);
        const float jy = m[2] + 0.5f * (Fo.fy + rho * kp.gy);
        const float jz = m[3] + 0.5f * (Fo.fz + rho * kp.gz);
        const float inv = 1.0f / rho;
        if (rho_out) rho_out[c.idx] = rho;
        if (u_out) {
            u_out[c.idx] = jx * inv;
            u_out[kp.ncell + c.idx] = jy * inv;
            u_out[2 * kp.ncell + c.idx] = jz * inv;
        }
        acc[0] = rho;
        acc[1] = jx;
        acc[2] = jy;
        acc[3] = jz;
    } else if (inside) {
        if (rho_out) rho_out[c.idx] = 0.0f;
        if (u_out) {
            u_out[c.idx] = 0.0f;
            u_out[kp.ncell + c.idx] = 0.0f;
            u_out[2 * kp.ncell + c.idx] = 0.0f;
        }
    }
    // fixed-order block reduction in FP64: warp tree, then warps in order
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((tid & 31) == 0) red[k][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < 4) {
        double s = 0.0;
        for (int w = 0; w < CS_BX * CS_BY * CS_BZ / 32; ++w) s += red[tid][w];
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        partials[4 * b + tid] = s;
    }
}

// ---- checkpoint gather: populations of the current state in natural order
template <int PARITY, bool SOLIDS, bool F16>
__global__ void gather_kernel(KParams kp, const void* __restrict__ fv, const uint32_t* __restrict__ nbmask,
                              float* __restrict__ out, const float* __restrict__ rsrc) {
    using T = typename std::conditional<F16, __half, float>::type;
    const T* f = reinterpret_cast<const T*>(fv);
    const int x = blockIdx.x * PSI_BX + threadIdx.x;
    const int y = blockIdx.y * PSI_BY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= kp.nx || y >= kp.ny) return;
    const Cell c = make_cell(kp, x, y, z);
    const uint32_t bits = SOLIDS ? solid_bits<Q>(kp, nbmask, c) : 0u;
    float p[Q];
    if (bits & 1u) {
#pragma unroll
        for (int i = 0; i < Q; ++i) p[i] = 0.0f;
    } else {
        gather<Q, PARITY, SOLIDS>(kp, f, c, bits, p);
        if (F16) denorm<Q, SOLIDS>(p, bits, RsCell{rsrc, c});
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) out[i * kp.ncell + c.idx] = p[i];
}

// ---- contact detector (Sec. III E, Sec. IV B): liquid fluid cells (rho > thr) with a solid
// lattice neighbour (mask or wall), and the liquid footprint in the layer z = 0 above a bottom
// wall.  out[0] += such cells, out[1] += liquid cells of the floor layer, out[2..5] = min / max
// of their x and y.  rho is formed as the moments kernel forms it.
constexpr int CT_BX = 32, CT_BY = 8;
template <int PARITY, bool F16>
__global__ void __launch_bounds__(CT_BX * CT_BY) contact_kernel(KParams kp, const void* __restrict__ fv,
                                                              const uint32_t* __restrict__ nbmask, float thr,
                                                              int* __restrict__ out, const float* __restrict__ rsrc) {
    using T = typename std::conditional<F16, __half, float>::type;
    const T* f = reinterpret_cast<const T*>(fv);
    const int x = blockIdx.x * CT_BX + threadIdx.x;
    const int y = blockIdx.y * CT_BY + threadIdx.y;
    const int z = blockIdx.z;
    bool wet = false;
    if (x < kp.nx && y < kp.ny) {
        const Cell c = make_cell(kp, x, y, z);
        const uint32_t bits = solid_bits<Q>(kp, nbmask, c);
        if (!(bits & 1u) && bits != 0u) {
            float p[Q], m[Q];
            gather<Q, PARITY, true>(kp, f, c, bits, p);
            if (F16) denorm<Q, true>(p, bits, RsCell{rsrc, c});
            to_moments<Q>(p, m);
            wet = m[0] > thr;
        }
    }
    const bool on_floor = wet && kp.wall_z && z == 0;
    const int nwet = __syncthreads_count(wet);
    const int nfloor = __syncthreads_count(on_floor);
    if (nfloor) {
        const unsigned lane_any = __ballot_sync(0xffffffffu, on_floor);
        const int xmin = __reduce_min_sync(0xffffffffu, on_floor ? x : INT_MAX);
        const int xmax = __reduce_max_sync(0xffffffffu, on_floor ? x : INT_MIN);
        const int ymin = __reduce_min_sync(0xffffffffu, on_floor ? y : INT_MAX);
        const int ymax = __reduce_max_sync(0xffffffffu, on_floor ? y : INT_MIN);
        if (lane_any && (threadIdx.x & 31) == 0) {
            atomicMin(out + 2, xmin);
            atomicMax(out + 3, xmax);
            atomicMin(out + 4, ymin);
            atomicMax(out + 5, ymax);
        }
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        if (nwet) atomicAdd(out, nwet);
        if (nfloor) atomicAdd(out + 1, nfloor);
    }
}

dim3 psi_grid(const KParams& kp) {
    return dim3((kp.nx + PSI_BX - 1) / PSI_BX, (kp.ny + PSI_BY - 1) / PSI_BY, kp.nz);
}
dim3 cs_grid(const KParams& kp) {
    return dim3((kp.nx + CS_BX - 1) / CS_BX, (kp.ny + CS_BY - 1) / CS_BY, (kp.nz + CS_BZ - 1) / CS_BZ);
}

// Launches one collide_kernel instantiation (internal linkage: each lattice's translation unit
// must launch its own kernels).  LBM_ZM_CARVEOUT >= 0 sets the preferred shared-memory carveout
// (percent) once; the default leaves the driver's choice, which keeps L1 large for the
// neighbour and psi-halo loads.
#ifndef LBM_ZM_CARVEOUT
#define LBM_ZM_CARVEOUT -1
#endif
template <int PARITY, bool SOLIDS, bool MULTIPHASE, bool F16>
cudaError_t launch_collide_variant(dim3 g, dim3 b, cudaStream_t st, const KParams& kp, const Bufs& B, int zc) {
    if (LBM_ZM_CARVEOUT >= 0) {
        static bool configured = false;
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(collide_kernel<PARITY, SOLIDS, MULTIPHASE, F16>,
                                                 cudaFuncAttributePreferredSharedMemoryCarveout, LBM_ZM_CARVEOUT);
            if (e != cudaSuccess) return e;
            configured = true;
        }
    }
    collide_kernel<PARITY, SOLIDS, MULTIPHASE, F16><<<g, b, 0, st>>>(kp, B.psi, B.nbmask, B.status, zc, B.rsrc, B.rnew);
    return cudaGetLastError();
}

template <bool F16>
cudaError_t launch_collide_store(dim3 g, dim3 b, cudaStream_t st, const KParams& kp, const Bufs& B, int zc, int key) {
    switch (key) {
        case 0: return launch_collide_variant<0, false, false, F16>(g, b, st, kp, B, zc);
        case 1: return launch_collide_variant<0, false, true, F16>(g, b, st, kp, B, zc);
        case 2: return launch_collide_variant<0, true, false, F16>(g, b, st, kp, B, zc);
        case 3: return launch_collide_variant<0, true, true, F16>(g, b, st, kp, B, zc);
        case 4: return launch_collide_variant<1, false, false, F16>(g, b, st, kp, B, zc);
        case 5: return launch_collide_variant<1, false, true, F16>(g, b, st, kp, B, zc);
        case 6: return launch_collide_variant<1, true, false, F16>(g, b, st, kp, B, zc);
        default: return launch_collide_variant<1, true, true, F16>(g, b, st, kp, B, zc);
    }
}

template <bool F16>
void launch_psi_store(dim3 g, dim3 b, cudaStream_t st, const KParams& kp, int parity, int solids, const Bufs& B) {
    if (parity == 2) psi_kernel<2, false, F16><<<g, b, 0, st>>>(kp, B.psi, B.nbmask, B.status, B.rsrc, B.rnew);
    else if (parity == 0 && !solids) psi_kernel<0, false, F16><<<g, b, 0, st>>>(kp, B.psi, B.nbmask, B.status, B.rsrc, B.rnew);
    else if (parity == 0) psi_kernel<0, true, F16><<<g, b, 0, st>>>(kp, B.psi, B.nbmask, B.status, B.rsrc, B.rnew);
    else if (!solids) psi_kernel<1, false, F16><<<g, b, 0, st>>>(kp, B.psi, B.nbmask, B.status, B.rsrc, B.rnew);
    else psi_kernel<1, true, F16><<<g, b, 0, st>>>(kp, B.psi, B.nbmask, B.status, B.rsrc, B.rnew);
}

template <bool F16>
void launch_moments_store(dim3 g, dim3 b, cudaStream_t st, const KParams& kp, int key, const Bufs& B, float* rho,
                          float* u, double* partials) {
    switch (key) {
        case 0: moments_kernel<0, false, false, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
        case 1: moments_kernel<0, false, true, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
        case 2: moments_kernel<0, true, false, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
        case 3: moments_kernel<0, true, true, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
        case 4: moments_kernel<1, false, false, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
        case 5: moments_kernel<1, false, true, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
        case 6: moments_kernel<1, true, false, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
        default: moments_kernel<1, true, true, F16><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, B.rsrc); break;
    }
}

template <bool F16>
void launch_gather_store(dim3 g, dim3 b, cudaStream_t st, const KParams& kp, int parity, int solids, const Bufs& B,
                         float* out) {
    if (parity == 2) gather_kernel<2, false, F16><<<g, b, 0, st>>>(kp, B.f, B.nbmask, out, B.rsrc);
    else if (parity == 0 && !solids) gather_kernel<0, false, F16><<<g, b, 0, st>>>(kp, B.f, B.nbmask, out, B.rsrc);
    else if (parity == 0) gather_kernel<0, true, F16><<<g, b, 0, st>>>(kp, B.f, B.nbmask, out, B.rsrc);
    else if (!solids) gather_kernel<1, false, F16><<<g, b, 0, st>>>(kp, B.f, B.nbmask, out, B.rsrc);
    else gather_kernel<1, true, F16><<<g, b, 0, st>>>(kp, B.f, B.nbmask, out, B.rsrc);
}

// multi-domain launch helpers (internal linkage: each lattice's translation unit launches its own kernels)
template <int S>
cudaError_t launch_collide_batch_shape(const KParams& phys, const BatchDomTable& doms, const BatchTile* tiles,
                                       int ntiles, int key, cudaStream_t st) {
    const dim3 b(BATCH_SHAPES[S].bx, BATCH_SHAPES[S].by);
    switch (key) {
        case 0: collide_batch_kernel<0, false, false, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
        case 1: collide_batch_kernel<0, false, true, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
        case 2: collide_batch_kernel<0, true, false, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
        case 3: collide_batch_kernel<0, true, true, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
        case 4: collide_batch_kernel<1, false, false, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
        case 5: collide_batch_kernel<1, false, true, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
        case 6: collide_batch_kernel<1, true, false, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
        default: collide_batch_kernel<1, true, true, S><<<ntiles, b, 0, st>>>(phys, doms, tiles); break;
    }
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_psi_batch_shape(const KParams& phys, const BatchDomTable& doms, const BatchTile* tiles, int ntiles,
                                   int parity, int solids, cudaStream_t st) {
    const dim3 b(BATCH_SHAPES[S].bx, BATCH_SHAPES[S].by);
    if (parity == 0 && !solids) psi_batch_kernel<0, false, S><<<ntiles, b, 0, st>>>(phys, doms, tiles);
    else if (parity == 0) psi_batch_kernel<0, true, S><<<ntiles, b, 0, st>>>(phys, doms, tiles);
    else if (!solids) psi_batch_kernel<1, false, S><<<ntiles, b, 0, st>>>(phys, doms, tiles);
    else psi_batch_kernel<1, true, S><<<ntiles, b, 0, st>>>(phys, doms, tiles);
    return cudaGetLastError();
}

}  // namespace

#define LBM_CAT2(a, b) a##b
#define LBM_CAT(a, b) LBM_CAT2(a, b)

cudaError_t LBM_CAT(launch_psi_q, LBM_Q)(const KParams& kp, int parity, int solids, const Bufs& B, cudaStream_t st) {
    if (B.paired) {
        const dim3 g((kp.hx + PSI_BX - 1) / PSI_BX, (kp.ny + PSI_BY - 1) / PSI_BY, kp.nz), b(PSI_BX, PSI_BY);
        if (parity == 0 && !solids) psi_pair_kernel<0, false><<<g, b, 0, st>>>(kp, B.psi, B.status, B.rsrc, B.rnew);
        else if (parity == 0) psi_pair_kernel<0, true><<<g, b, 0, st>>>(kp, B.psi, B.status, B.rsrc, B.rnew);
        else if (!solids) psi_pair_kernel<1, false><<<g, b, 0, st>>>(kp, B.psi, B.status, B.rsrc, B.rnew);
        else psi_pair_kernel<1, true><<<g, b, 0, st>>>(kp, B.psi, B.status, B.rsrc, B.rnew);
        return cudaGetLastError();
    }
    const dim3 g = psi_grid(kp), b(PSI_BX, PSI_BY);
    if (B.f16) launch_psi_store<true>(g, b, st, kp, parity, solids, B);
    else launch_psi_store<false>(g, b, st, kp, parity, solids, B);
    return cudaGetLastError();
}

// z planes per block: enough blocks for a few waves of resident blocks on 152 SMs
// z-planes per block of the z-marching kernels.  Blocks of equal size run in waves of
// (SMs x resident blocks); a last wave that is mostly empty leaves SMs idle, and every chunk
// costs about h planes' worth of extra time at its start (the psi planes below and at its first
// plane, the first loads with nothing to overlap them); and blocks differ in duration, which more
// waves even out.  Over the chunk counts that give at least three waves, the choice minimises
// (1 + h / zc) x ceil(waves) / waves x (1 + 0.2 / waves) (0.2 fitted to 256^3 sweeps).
static int choose_zchunk(const KParams& kp, double h, int nz, int by, int minb) {
    if (kp.zchunk > 0) return kp.zchunk < nz ? kp.zchunk : nz;
    if (nz <= 1) return 1;
    static const int sms = [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || n <= 0)
            n = 152;
        return n;
    }();
    thread_local long long key[4] = {-1, -1, -1, -1};
    thread_local int cached = 1;
    const long long k[4] = {kp.nx, kp.ny, nz, (long long)(h * 1024.0) + 4096LL * (by + 64LL * minb)};
    if (k[0] == key[0] && k[1] == key[1] && k[2] == key[2] && k[3] == key[3]) return cached;
    const double cap = (double)sms * minb;
    const long long cols = (long long)((kp.nx + ZM_BX - 1) / ZM_BX) * ((kp.ny + by - 1) / by);
    int best = nz;
    double best_cost = 1e300;
    for (int c = 1; c <= nz; ++c) {
        const int zc = (nz + c - 1) / c;
        const int chunks = (nz + zc - 1) / zc;
        if (chunks != c) continue;                 // the same split as a smaller count
        const double waves = (double)(cols * chunks) / cap;
        if (waves < 3.0 && c < nz) continue;
        const double cost = (1.0 + h / zc) * std::ceil(waves) / waves * (1.0 + 0.2 / waves);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = zc; }
    }
    for (int i = 0; i < 4; ++i) key[i] = k[i];
    cached = best;
    return best;
}

// over the planes [zlo, zhi) the whole-grid collide kernels march through
static int collide_zchunk(const KParams& kp) { return choose_zchunk(kp, 1.0, kp.zhi - kp.zlo, ZM_BY, ZM_MINB); }

cudaError_t LBM_CAT(launch_collide_q, LBM_Q)(const KParams& kp, int parity, int solids, const Bufs& B,
                                             cudaStream_t st) {
    if (B.paired) {
        // tiles of 32 pairs: the z-chunk choice counts columns of hx words
        KParams kw = kp;
        kw.nx = kp.hx;
        const int planes = kp.zhi - kp.zlo;
        const int zc = choose_zchunk(kw, 1.0, planes, PR_BY, PR_MINB);
        const dim3 g((kp.hx + PR_BX - 1) / PR_BX, (kp.ny + PR_BY - 1) / PR_BY, (planes + zc - 1) / zc), b(PR_BX, PR_BY);
        const int key = parity * 4 + (solids ? 2 : 0) + (kp.multiphase ? 1 : 0);
        const float* r0 = B.rsrc;
        const float* r1 = B.rnew;
        switch (key) {
            case 0: collide_pair_kernel<0, false, false><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
            case 1: collide_pair_kernel<0, false, true><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
            case 2: collide_pair_kernel<0, true, false><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
            case 3: collide_pair_kernel<0, true, true><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
            case 4: collide_pair_kernel<1, false, false><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
            case 5: collide_pair_kernel<1, false, true><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
            case 6: collide_pair_kernel<1, true, false><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
            default: collide_pair_kernel<1, true, true><<<g, b, 0, st>>>(kp, B.psi, B.status, zc, r0, r1); break;
        }
        return cudaGetLastError();
    }
    const int zc = collide_zchunk(kp);
    const int planes = kp.zhi - kp.zlo;
    const dim3 g((kp.nx + ZM_BX - 1) / ZM_BX, (kp.ny + ZM_BY - 1) / ZM_BY, (planes + zc - 1) / zc), b(ZM_BX, ZM_BY);
    const int key = parity * 4 + (solids ? 2 : 0) + (kp.multiphase ? 1 : 0);
    return B.f16 ? launch_collide_store<true>(g, b, st, kp, B, zc, key)
                 : launch_collide_store<false>(g, b, st, kp, B, zc, key);
}

cudaError_t LBM_CAT(launch_collide_batch_q, LBM_Q)(const KParams& phys, const BatchDomTable& doms,
                                                   const BatchTile* tiles, int ntiles, int parity, int solids,
                                                   int shape, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    const int key = parity * 4 + (solids ? 2 : 0) + (phys.multiphase ? 1 : 0);
    switch (shape) {
        case 0: return launch_collide_batch_shape<0>(phys, doms, tiles, ntiles, key, st);
        case 1: return launch_collide_batch_shape<1>(phys, doms, tiles, ntiles, key, st);
        case 2: return launch_collide_batch_shape<2>(phys, doms, tiles, ntiles, key, st);
        case 3: return launch_collide_batch_shape<3>(phys, doms, tiles, ntiles, key, st);
        case 4: return launch_collide_batch_shape<4>(phys, doms, tiles, ntiles, key, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t LBM_CAT(launch_psi_runs_q, LBM_Q)(const KParams& phys, const BatchDomTable& doms, const BatchRun* runs,
                                              int nruns, int parity, cudaStream_t st) {
    if (nruns <= 0) return cudaSuccess;
    if (parity == 0) psi_run_kernel<0><<<nruns, RUN_NT, 0, st>>>(phys, doms, runs);
    else psi_run_kernel<1><<<nruns, RUN_NT, 0, st>>>(phys, doms, runs);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_psi_batch_q, LBM_Q)(const KParams& phys, const BatchDomTable& doms,
                                               const BatchTile* tiles, int ntiles, int parity, int solids, int shape,
                                               cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    switch (shape) {
        case 0: return launch_psi_batch_shape<0>(phys, doms, tiles, ntiles, parity, solids, st);
        case 1: return launch_psi_batch_shape<1>(phys, doms, tiles, ntiles, parity, solids, st);
        case 2: return launch_psi_batch_shape<2>(phys, doms, tiles, ntiles, parity, solids, st);
        case 3: return launch_psi_batch_shape<3>(phys, doms, tiles, ntiles, parity, solids, st);
        case 4: return launch_psi_batch_shape<4>(phys, doms, tiles, ntiles, parity, solids, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t LBM_CAT(launch_contact_q, LBM_Q)(const KParams& kp, int parity, const Bufs& B, float thr, int* out,
                                             cudaStream_t st) {
    const dim3 g((kp.nx + CT_BX - 1) / CT_BX, (kp.ny + CT_BY - 1) / CT_BY, kp.nz), b(CT_BX, CT_BY);
    if (B.f16) {
        if (parity == 0) contact_kernel<0, true><<<g, b, 0, st>>>(kp, B.f, B.nbmask, thr, out, B.rsrc);
        else contact_kernel<1, true><<<g, b, 0, st>>>(kp, B.f, B.nbmask, thr, out, B.rsrc);
    } else {
        if (parity == 0) contact_kernel<0, false><<<g, b, 0, st>>>(kp, B.f, B.nbmask, thr, out, nullptr);
        else contact_kernel<1, false><<<g, b, 0, st>>>(kp, B.f, B.nbmask, thr, out, nullptr);
    }
    return cudaGetLastError();
}

// one-pass tiles: 32 x 4 cells (the 76-cell border fits the 128 threads), 7 (D3Q19) / 5 (D3Q27)
// blocks per SM -- the best of 32 x 4 / 8 / 16 tiles and 4-8 blocks per SM, measured
constexpr int OP_BY = 4, OP_MINB = LBM_Q == 19 ? 7 : 5;

cudaError_t LBM_CAT(launch_onepass_tma_q, LBM_Q)(const KParams& kp, const CUtensorMap& read_map, unsigned* status,
                                                 unsigned extra_tx, long long wait_cycles, cudaStream_t st) {
    // two staged planes at a chunk's start
    const int zc = choose_zchunk(kp, 2.0, kp.nz, 4, OT_MINB);
    const dim3 g(kp.nx / 32, kp.ny / 4, (kp.nz + zc - 1) / zc), b(32, 4);
    const size_t smem = sizeof(OtShared);
    static bool configured[2] = {false, false};
    cudaError_t e = cudaSuccess;
    if (kp.multiphase) {
        if (!configured[1]) {
            e = cudaFuncSetAttribute(collide_onepass_tma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            configured[1] = e == cudaSuccess;
        }
        if (e == cudaSuccess)
            collide_onepass_tma_kernel<true><<<g, b, smem, st>>>(kp, read_map, status, zc, extra_tx, wait_cycles);
    } else {
        if (!configured[0]) {
            e = cudaFuncSetAttribute(collide_onepass_tma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            configured[0] = e == cudaSuccess;
        }
        if (e == cudaSuccess)
            collide_onepass_tma_kernel<false><<<g, b, smem, st>>>(kp, read_map, status, zc, extra_tx, wait_cycles);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t LBM_CAT(launch_onepass_q, LBM_Q)(const KParams& kp, unsigned* status, cudaStream_t st) {
    // a chunk starts with two psi planes whose loads nothing overlaps
    const int zc = choose_zchunk(kp, 1.5, kp.nz, OP_BY, OP_MINB);
    const dim3 g((kp.nx + 31) / 32, (kp.ny + OP_BY - 1) / OP_BY, (kp.nz + zc - 1) / zc), b(32, OP_BY);
    if (kp.multiphase) collide_onepass_kernel<true, OP_BY, OP_MINB><<<g, b, 0, st>>>(kp, status, zc);
    else collide_onepass_kernel<false, OP_BY, OP_MINB><<<g, b, 0, st>>>(kp, status, zc);
    return cudaGetLastError();
}

unsigned long long LBM_CAT(bounds_violations_q, LBM_Q)() {
#if LBM_BOUNDS_CHECK
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, lbm_bounds_count, sizeof(v)) != cudaSuccess) return ~0ull;
    return v;
#else
    return 0;
#endif
}

cudaError_t LBM_CAT(launch_pull_store_q, LBM_Q)(const KParams& kp, const float* fin, long long fstride, float* fout,
                                                cudaStream_t st) {
    const long long blocks = (kp.ncell + 255) / 256;
    const int g = (int)(blocks < 152LL * 64 ? blocks : 152LL * 64);
    pull_store_kernel<<<g, 256, 0, st>>>(kp, fin, fstride, fout);
    return cudaGetLastError();
}


cudaError_t LBM_CAT(launch_init_q, LBM_Q)(const KParams& kp, const Bufs& B, const float* rho, const float* u,
                                          cudaStream_t st) {
    const long long blocks = (kp.ncell + 255) / 256;
    const int g = (int)(blocks < 152LL * 64 ? blocks : 152LL * 64);
    if (B.f16) init_kernel<true><<<g, 256, 0, st>>>(kp, B.f, rho, u, B.nbmask, const_cast<float*>(B.rsrc));
    else init_kernel<false><<<g, 256, 0, st>>>(kp, B.f, rho, u, B.nbmask, nullptr);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_f16_restore_q, LBM_Q)(const KParams& kp, const Bufs& B, const float* fin, cudaStream_t st) {
    const long long blocks = (kp.ncell + 255) / 256;
    const int g = (int)(blocks < 152LL * 64 ? blocks : 152LL * 64);
    float* r = const_cast<float*>(B.rsrc);
    f16_density_kernel<<<g, 256, 0, st>>>(kp, fin, B.nbmask, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    f16_pack_kernel<<<g, 256, 0, st>>>(kp, fin, B.nbmask, r, reinterpret_cast<__half*>(B.f));
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_moments_q, LBM_Q)(const KParams& kp, int parity, int solids, const Bufs& B, float* rho,
                                             float* u, double* partials, int* nblocks, cudaStream_t st) {
    const dim3 g = cs_grid(kp), b(CS_BX, CS_BY, CS_BZ);
    *nblocks = (int)(g.x * g.y * g.z);
    if (parity == 2) {   // one-pass layout (FP32, no solids)
        if (kp.multiphase)
            moments_kernel<2, false, true, false><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, nullptr);
        else
            moments_kernel<2, false, false, false><<<g, b, 0, st>>>(kp, B.f, B.psi, B.nbmask, rho, u, partials, nullptr);
        return cudaGetLastError();
    }
    const int key = parity * 4 + (solids ? 2 : 0) + (kp.multiphase ? 1 : 0);
    if (B.f16) launch_moments_store<true>(g, b, st, kp, key, B, rho, u, partials);
    else launch_moments_store<false>(g, b, st, kp, key, B, rho, u, partials);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_gather_q, LBM_Q)(const KParams& kp, int parity, int solids, const Bufs& B, float* out,
                                            cudaStream_t st) {
    const dim3 g = psi_grid(kp), b(PSI_BX, PSI_BY);
    if (B.f16) launch_gather_store<true>(g, b, st, kp, parity, solids, B, out);
    else launch_gather_store<false>(g, b, st, kp, parity, solids, B, out);
    return cudaGetLastError();
}

}  // namespace lbm
