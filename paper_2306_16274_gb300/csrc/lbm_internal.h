// Internal interface between the C ABI (capi.cu) and the per-lattice kernel
// translation units (kernels_q19.cu, kernels_q27.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Status bits raised by kernels (read by lbm_sync).
enum : unsigned { ST_UNSTABLE = 1u, ST_EOS_RANGE = 2u, ST_TIMEOUT = 4u };

// Everything a kernel needs, flattened to floats on the host (derived terms
// precomputed in double, rounded once).
struct KParams {
    int nx, ny, nz;
    int wall_x, wall_y, wall_z;   // 1 = half-way bounce-back walls on that axis
    long long plane;              // stride between population planes (floats), >= ncell
    long long ncell;              // nx * ny * nz
    int multiphase;               // EOS present (psi, F_int, F_ads, Q, sigma term)
    int eos;                      // 1 Carnahan-Starling, 2 piecewise linear
    // Carnahan-Starling: p = rho RT g(eta) - a rho^2, eta = (b/4) rho
    float cs_a, cs_b4, cs_RT;
    float2 cs_a_ff, cs_b4_ff, cs_RT_ff;   // the same as float-float pairs (hi, lo)
    float2 third_ff;              // 1/3 = c_s^2 as a float-float pair
    float psi_ext_rho;            // rho >= this: evaluate the EOS and p - rho c_s^2 in float-float
    // piecewise linear (Eq. e19)
    float pw_rho1, pw_rho2, pw_tv, pw_tm, pw_tl, pw_p1, pw_p2;
    float two_over_G;             // psi^2 = (2/G)(p_EOS - rho c_s^2)
    float2 two_over_G_ff;
    float G;                      // Eq. e15
    float G_ads;                  // Sec. III E
    float kappa_G_half;           // kappa G / 2 of Eq. e18
    float sigma_coef;             // 6 sigma G^2 / (1/s_e - 1/2): |F_int|^2 / psi^2 = G^2 |S|^2
    float q7_coef;                // 4 / (5 (1/s_e - 1/2))
    float s[10];                  // s0 s1 s2 s2b s3 s3b s4 s4b s5 s6
    float c[10];                  // 1 - s/2
    float inv_tnu;                // 1 / (1/s2 - 1/2)
    int variable_nu;
    float nu_v, dnu_drho, rho_v;  // nu(rho) = nu_v + dnu_drho (rho - rho_v)
    float gx, gy, gz;             // body force per unit mass
    float* fq[27];                // base of population plane i (f + i * plane); cells < 2^31
    int zchunk;                   // z planes per collide block (0 = automatic)
    int zlo, zhi;                 // planes [zlo, zhi) the whole-grid collide kernels march through
    float* gq[27];                // one-pass layout: planes of the copy the step writes
    // shifted FP16 store in the x-paired layout (even nx, x periodic, no solid mask): word w of a
    // row holds cells w (low half) and w + hx (high half), hx = nx / 2, so a shift by one cell in
    // x moves both cells of a word to one other word
    int paired;
    int hx;
};

// Geometry and device buffers of one member of a multi-domain launch (its physics come from the
// group's KParams, passed by value).
struct BatchDom {
    int nx, ny, nz, wall_x, wall_y, wall_z;
    long long plane;
    float* base;                  // population plane 0; plane i at base + i * plane
    float* psi;
    const uint32_t* nbmask;
    unsigned* status;
    uint32_t mx, my;              // n / nx and n / ny as (n * m) >> s for n < 2^31 (div_magic)
    int sx, sy;
};

// Division by an invariant d in [1, 2^31) as a multiply and a shift (Granlund and Montgomery, PLDI
// 1994, Thm. 4.2, with N = 31): l = ceil(log2 d), m = ceil(2^(31 + l) / d), s = 31 + l; then
// floor(n / d) = (n * m) >> s for every n < 2^31, and m < 2^32.
inline void div_magic(uint32_t d, uint32_t& m, int& s) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    m = (uint32_t)(((1ull << (31 + l)) + d - 1) / d);
    s = 31 + l;
}

// A run of cells [begin, end) of member d of a multi-domain launch (cell index (z ny + y) nx + x),
// none of which needs solid handling: the density/psi pass covers whole planes of a member this way,
// one block per run, with no lanes left idle at the ends of rows.
struct BatchRun {
    int d;
    uint32_t begin, end;
};

// Members of one multi-domain launch.  The table travels in the kernel parameters (constant bank),
// so a block's member addresses are read like the single-domain kernel's plane pointers.
constexpr int BATCH_LAUNCH_DOMS = 64;
struct BatchDomTable {
    BatchDom d[BATCH_LAUNCH_DOMS];
};

// One block of a multi-domain launch: member d of the launch's table, cells [x0, x0+tile width) x
// [y0, y0+tile height) x [z0, z0+zc) (clipped to the domain).  narrow = 1: the tile is
// BATCH_NARROW_BX cells wide and (threads / BATCH_NARROW_BX) high instead of the launch's shape --
// the last columns of rows whose length leaves at most that many cells past the last full tile.
constexpr int BATCH_NARROW_BX = 16;
struct BatchTile {
    int d, x0, y0, z0, zc, narrow;
};

// Tile shapes of the multi-domain kernels, compiled for each lattice; lbm_batch_tune picks one per
// group.  Width and height of a tile in cells (one thread each) and the resident blocks per SM the
// collide kernel is compiled for on D3Q19 / D3Q27 (its register budget).  Narrower tiles waste fewer
// lanes on domains whose x extent is not a multiple of 32; lower residency leaves more registers.
struct BatchShape {
    int bx, by, minb19, minb27;
};
constexpr int BATCH_NSHAPES = 5;
constexpr BatchShape BATCH_SHAPES[BATCH_NSHAPES] = {
    {32, 4, 7, 5}, {32, 2, 14, 10}, {16, 8, 7, 5}, {16, 4, 14, 10}, {32, 4, 6, 4}};

// Device buffers of one context's launches.  f: the population slots, floats or (f16) the
// shifted FP16 store; rsrc: the densities the stored slots were written with; rnew: the other
// density buffer (the density pass writes it, the collide pass writes relative to it).
struct Bufs {
    void* f;
    float* psi;
    const uint32_t* nbmask;
    unsigned* status;
    int f16;
    int paired;                   // f16 in the x-paired layout (KParams::paired)
    const float* rsrc;
    float* rnew;
};

// Launchers (one set per lattice).  parity: 0 = natural layout (even AA step),
// 1 = swapped layout (odd AA step).  solids: walls or a solid mask exist.
#define LBM_DECLARE_LAUNCHERS(Q)                                                                    \
    cudaError_t launch_psi_q##Q(const KParams& kp, int parity, int solids, const Bufs& B,           \
                                cudaStream_t st);                                                   \
    cudaError_t launch_collide_q##Q(const KParams& kp, int parity, int solids, const Bufs& B,       \
                                    cudaStream_t st);                                               \
    cudaError_t launch_init_q##Q(const KParams& kp, const Bufs& B, const float* rho, const float* u, \
                                 cudaStream_t st);                                                  \
    cudaError_t launch_f16_restore_q##Q(const KParams& kp, const Bufs& B, const float* fin,         \
                                        cudaStream_t st);                                           \
    cudaError_t launch_moments_q##Q(const KParams& kp, int parity, int solids, const Bufs& B,       \
                                    float* rho, float* u, double* partials, int* nblocks,            \
                                    cudaStream_t st);                                               \
    cudaError_t launch_gather_q##Q(const KParams& kp, int parity, int solids, const Bufs& B,        \
                                   float* out, cudaStream_t st);                                     \
    cudaError_t launch_collide_batch_q##Q(const KParams& phys, const BatchDomTable& tab,             \
                                          const BatchTile* tiles, int ntiles, int parity, int solids,  \
                                          int shape, cudaStream_t st);                                \
    cudaError_t launch_psi_batch_q##Q(const KParams& phys, const BatchDomTable& tab,                 \
                                      const BatchTile* tiles, int ntiles, int parity, int solids,      \
                                      int shape, cudaStream_t st);                                    \
    cudaError_t launch_psi_runs_q##Q(const KParams& phys, const BatchDomTable& tab, const BatchRun* runs, \
                                     int nruns, int parity, cudaStream_t st);                          \
    cudaError_t launch_contact_q##Q(const KParams& kp, int parity, const Bufs& B, float thr, int* out, \
                                    cudaStream_t st);                                               \
    cudaError_t launch_onepass_q##Q(const KParams& kp, unsigned* status, cudaStream_t st);          \
    cudaError_t launch_onepass_tma_q##Q(const KParams& kp, const CUtensorMap& read_map, unsigned* status, \
                                        unsigned extra_tx, long long wait_cycles, cudaStream_t st);       \
    cudaError_t launch_pull_store_q##Q(const KParams& kp, const float* fin, long long fstride,       \
                                       float* fout, cudaStream_t st);                               \
    unsigned long long bounds_violations_q##Q();

LBM_DECLARE_LAUNCHERS(19)
LBM_DECLARE_LAUNCHERS(27)

// Lattice-independent kernels (capi.cu)
cudaError_t launch_nbmask(const KParams& kp, int Q, const uint8_t* solid, uint32_t* nbmask, cudaStream_t st);
cudaError_t launch_finish_sums(const double* partials, int nblocks, double* sums, cudaStream_t st);
cudaError_t launch_contact_init(int* out, cudaStream_t st);   // out[6] = 0, 0, INT_MAX, INT_MIN, INT_MAX, INT_MIN

// Sets the message lbm_last_error(NULL) returns on this thread (context-free entry points).
void set_thread_error(const char* msg);

// Number of blocks launch_moments_q* uses for partial sums (upper bound for the scratch size).
long long moments_partial_blocks(const KParams& kp);

}  // namespace lbm
