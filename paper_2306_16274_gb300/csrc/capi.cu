// C ABI of liblbm.so (declared in include/lbm.h): context lifetime, parameter
// validation and derivation, step sequencing (AA parity), host<->device
// marshalling, status handling and kernel timing.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "ctx_internal.h"

using lbm::KParams;

namespace {

thread_local std::string g_create_error;

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

#define CK(ctx, call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

bool rate_ok(double s) { return s > 0.0 && s < 2.0 && std::isfinite(s); }

lbm_status validate(const lbm_params* p, std::string& why) {
    if (!p) { why = "params is NULL"; return LBM_ERR_ARG; }
    if (p->lattice != 19 && p->lattice != 27) { why = "lattice must be 19 or 27"; return LBM_ERR_ARG; }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { why = "nx, ny, nz must be >= 1"; return LBM_ERR_ARG; }
    if (p->nx > LBM_MAX_EXTENT || p->ny > LBM_MAX_EXTENT || p->nz > LBM_MAX_EXTENT) {
        why = "nx, ny, nz must be <= LBM_MAX_EXTENT (65535)";
        return LBM_ERR_ARG;
    }
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n >= (1LL << 31)) { why = "domain too large: at most 2^31 - 1 cells"; return LBM_ERR_ARG; }
    for (int a = 0; a < 3; ++a)
        if (p->bc[a] != LBM_BC_PERIODIC && p->bc[a] != LBM_BC_WALL) { why = "bc must be 0 or 1"; return LBM_ERR_ARG; }
    for (int k = 0; k < 10; ++k)
        if (!rate_ok(p->s[k])) { why = "relaxation rates must lie in (0, 2)"; return LBM_ERR_ARG; }
    if (p->eos != LBM_EOS_NONE && p->eos != LBM_EOS_CS && p->eos != LBM_EOS_PIECEWISE) {
        why = "unknown eos";
        return LBM_ERR_ARG;
    }
    if (p->eos != LBM_EOS_NONE) {
        if (!(p->G != 0.0) || !std::isfinite(p->G)) { why = "a multiphase EOS needs a finite G != 0"; return LBM_ERR_ARG; }
        if (p->eos == LBM_EOS_CS && !(p->eos_p[1] > 0.0 && p->eos_p[2] > 0.0 && p->eos_p[3] > 0.0)) {
            why = "Carnahan-Starling needs b, R, T > 0";
            return LBM_ERR_ARG;
        }
        if (p->eos == LBM_EOS_PIECEWISE && !(p->eos_p[0] > 0.0 && p->eos_p[1] > p->eos_p[0])) {
            why = "piecewise EOS needs 0 < rho1 < rho2";
            return LBM_ERR_ARG;
        }
    }
    if (p->zchunk < 0) { why = "zchunk must be >= 0"; return LBM_ERR_ARG; }
    if (p->store != LBM_STORE_FP32 && p->store != LBM_STORE_FP16) {
        why = "store must be LBM_STORE_FP32 or LBM_STORE_FP16";
        return LBM_ERR_ARG;
    }
    if (p->onepass < 0 || p->onepass > 2) { why = "onepass must be 0, 1 or 2 (LBM_ONEPASS_STAGED)"; return LBM_ERR_ARG; }
    if (p->onepass == 2 && (p->nx % 32 != 0 || p->ny % 4 != 0)) {
        why = "onepass = 2 (staged) needs nx a multiple of 32 and ny a multiple of 4";
        return LBM_ERR_ARG;
    }
    if (p->store_layout != LBM_LAYOUT_AUTO && p->store_layout != LBM_LAYOUT_SINGLE) {
        why = "store_layout must be LBM_LAYOUT_AUTO or LBM_LAYOUT_SINGLE";
        return LBM_ERR_ARG;
    }
    if (p->onepass && (p->store != LBM_STORE_FP32 || p->bc[0] != LBM_BC_PERIODIC || p->bc[1] != LBM_BC_PERIODIC ||
                       p->bc[2] != LBM_BC_PERIODIC)) {
        why = "onepass needs the FP32 store and periodic boundaries on all axes";
        return LBM_ERR_ARG;
    }
    if (p->variable_nu) {
        if (!(p->rho_l != p->rho_v) || !(p->nu_l > 0.0) || !(p->nu_v > 0.0)) {
            why = "variable viscosity needs rho_l != rho_v and nu_l, nu_v > 0";
            return LBM_ERR_ARG;
        }
    }
    return LBM_OK;
}

// d as an unevaluated float pair: hi = d rounded to float, lo = the remainder rounded to float
float2 ff_split(double d) {
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}

KParams derive(const lbm_params& p, long long plane) {
    KParams k{};
    k.nx = p.nx;
    k.ny = p.ny;
    k.nz = p.nz;
    k.wall_x = p.bc[0] == LBM_BC_WALL;
    k.wall_y = p.bc[1] == LBM_BC_WALL;
    k.wall_z = p.bc[2] == LBM_BC_WALL;
    k.ncell = (long long)p.nx * p.ny * p.nz;
    k.plane = plane;
    k.multiphase = p.eos != LBM_EOS_NONE;
    k.eos = p.eos;
    if (p.eos == LBM_EOS_CS) {
        const double a = p.eos_p[0], b = p.eos_p[1], R = p.eos_p[2], T = p.eos_p[3];
        k.cs_a_ff = ff_split(a);
        k.cs_b4_ff = ff_split(b / 4.0);
        k.cs_RT_ff = ff_split(R * T);
        k.third_ff = ff_split(1.0 / 3.0);
        k.cs_a = (float)a;
        k.cs_b4 = (float)(b / 4.0);
        k.cs_RT = (float)(R * T);
        // default threshold of the float-float branch: the critical density b rho_c = 0.52177
        const double thr = p.psi_ext_rho < 0.0 ? 0.52177 / b : p.psi_ext_rho;
        k.psi_ext_rho = (float)thr;
    } else {
        k.psi_ext_rho = INFINITY;
    }
    if (p.eos == LBM_EOS_PIECEWISE) {
        k.pw_rho1 = (float)p.eos_p[0];
        k.pw_rho2 = (float)p.eos_p[1];
        k.pw_tv = (float)p.eos_p[2];
        k.pw_tm = (float)p.eos_p[3];
        k.pw_tl = (float)p.eos_p[4];
        const double p1 = p.eos_p[0] * p.eos_p[2];
        k.pw_p1 = (float)p1;
        k.pw_p2 = (float)(p1 + (p.eos_p[1] - p.eos_p[0]) * p.eos_p[3]);
    }
    const double G = k.multiphase ? p.G : 0.0;
    k.G = (float)G;
    k.G_ads = k.multiphase ? (float)p.G_ads : 0.0f;
    const double tg = G != 0.0 ? 2.0 / G : 0.0;
    k.two_over_G_ff = ff_split(tg);
    k.two_over_G = (float)tg;
    k.kappa_G_half = (float)(p.kappa * G / 2.0);
    const double t_e = 1.0 / p.s[3] - 0.5;    // s_e = s2b (rate of m_7)
    k.sigma_coef = (float)(k.multiphase ? 6.0 * p.sigma * G * G / t_e : 0.0);
    k.q7_coef = (float)(4.0 / (5.0 * t_e));
    for (int i = 0; i < 10; ++i) {
        k.s[i] = (float)p.s[i];
        k.c[i] = (float)(1.0 - 0.5 * p.s[i]);
    }
    k.inv_tnu = (float)(1.0 / (1.0 / p.s[2] - 0.5));
    k.variable_nu = p.variable_nu ? 1 : 0;
    if (p.variable_nu) {
        k.nu_v = (float)p.nu_v;
        k.rho_v = (float)p.rho_v;
        k.dnu_drho = (float)((p.nu_l - p.nu_v) / (p.rho_l - p.rho_v));
    }
    k.gx = (float)p.g[0];
    k.gy = (float)p.g[1];
    k.gz = (float)p.g[2];
    k.zchunk = p.zchunk;
    k.zlo = 0;
    k.zhi = p.nz;
    return k;
}

// The shifted FP16 store keeps two cells per 4-byte word (x-paired layout) when nx is even, x is
// periodic and there is no solid mask; the layout is fixed whenever all slots are rewritten
// (create, init_fields, set_populations keep it until the next init_fields).
void set_layout(lbm_ctx* c, bool with_mask) {
    c->paired = c->f16 && c->p.store_layout == LBM_LAYOUT_AUTO && c->kp.nx % 2 == 0 && !c->kp.wall_x && !with_mask;
    c->kp.paired = c->paired;
    c->kp.hx = c->kp.nx / 2;
}

bool has_solids(const lbm_ctx* c) {
    return c->nbmask != nullptr || c->kp.wall_x || c->kp.wall_y || c->kp.wall_z;
}

// The context's buffers as the launchers take them.  Shifted FP16 store: rbuf[rs] holds the
// densities the stored slots were written with, rbuf[rs ^ 1] the newest densities.
lbm::Bufs bufs(const lbm_ctx* c) {
    lbm::Bufs b;
    b.f = c->f;
    b.psi = c->psi;
    b.nbmask = c->nbmask;
    b.status = c->status;
    b.f16 = c->f16;
    b.paired = c->paired;
    b.rsrc = c->f16 ? c->rbuf[c->rs] : nullptr;
    b.rnew = c->f16 ? c->rbuf[c->rs ^ 1] : nullptr;
    return b;
}

// density (+ psi) pass; with the FP16 store it also writes the densities the next collide pass
// normalises with, so it runs for single-phase domains too
cudaError_t run_psi(lbm_ctx* c) {
    if (!c->kp.multiphase && !c->f16) return cudaSuccess;
    const int s = has_solids(c);
    return c->Q == 19 ? lbm::launch_psi_q19(c->kp, c->parity, s, bufs(c), c->stream)
                      : lbm::launch_psi_q27(c->kp, c->parity, s, bufs(c), c->stream);
}

// Tensor map of one population copy for the staged one-pass kernel: a 4-D array (x, y, z,
// population) of floats, boxes of 40 x 8 x 1 x 1 (plane strides are multiples of 256 bytes; rows of
// nx floats with nx a multiple of 32).  The encoder is taken from the driver through the runtime, so
// the library links no driver library.
bool encode_copy_map(CUtensorMap* m, const void* base, const KParams& k, int Q) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<Encode>(fn);
    }();
    if (!encode) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)k.nx, (cuuint64_t)k.ny, (cuuint64_t)k.nz, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {(cuuint64_t)k.nx * 4, (cuuint64_t)k.nx * k.ny * 4, (cuuint64_t)k.plane * 4};
    const cuuint32_t box[4] = {40, 8, 1, 1};
    const cuuint32_t step[4] = {1, 1, 1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, step,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// onepass = 2: staged copies (full 32 x 4 tiles, so every box starts on a 16-byte boundary); one
// tensor map per population copy.  False if the driver cannot encode them.
bool setup_staging(lbm_ctx* c) {
    const void* copies[2] = {c->f, c->f2};
    for (int k = 0; k < 2; ++k) {
        if (!encode_copy_map(&c->tmap[k], copies[k], c->kp, c->Q)) return false;
        c->tmap_base[k] = copies[k];
    }
    c->staged = 1;
    return true;
}

// one-pass layout: one launch per step, then the copies trade places
cudaError_t run_onepass(lbm_ctx* c) {
    cudaError_t e;
    if (c->staged) {
        const int k = c->tmap_base[0] == c->f ? 0 : 1;      // the copy this step reads
        // waits on staged copies give up after ~2 s (2^32 cycles); the timeout test uses ~10 ms and
        // expects bytes that no copy delivers
        const unsigned extra = c->stage_timeout_test ? 4096u : 0u;
        const long long cycles = c->stage_timeout_test ? 20000000LL : 4294967296LL;
        e = c->Q == 19 ? lbm::launch_onepass_tma_q19(c->kp, c->tmap[k], c->status, extra, cycles, c->stream)
                       : lbm::launch_onepass_tma_q27(c->kp, c->tmap[k], c->status, extra, cycles, c->stream);
    } else {
        e = c->Q == 19 ? lbm::launch_onepass_q19(c->kp, c->status, c->stream)
                       : lbm::launch_onepass_q27(c->kp, c->status, c->stream);
    }
    std::swap(c->f, c->f2);
    for (int i = 0; i < 27; ++i) std::swap(c->kp.fq[i], c->kp.gq[i]);
    return e;
}

// Walls only at the two z ends (the droplet-impact setup): the planes between them need no
// solid handling, so they take the solid-free kernel and only the two wall planes the solid one.
bool zwalls_only(const lbm_ctx* c) {
    return !c->nbmask && !c->kp.wall_x && !c->kp.wall_y && c->kp.wall_z && c->kp.nz >= 3 && !c->onepass;
}

cudaError_t launch_collide(const lbm_ctx* c, const lbm::KParams& k, int solids) {
    return c->Q == 19 ? lbm::launch_collide_q19(k, c->parity, solids, bufs(c), c->stream)
                      : lbm::launch_collide_q27(k, c->parity, solids, bufs(c), c->stream);
}

cudaError_t run_collide(lbm_ctx* c) {
    cudaError_t e;
    if (zwalls_only(c)) {
        // each slot is read and written by one cell only, so the three plane ranges are independent
        lbm::KParams k = c->kp;
        k.zlo = 1;
        k.zhi = k.nz - 1;
        e = launch_collide(c, k, 0);
        k.zlo = 0;
        k.zhi = 1;
        if (e == cudaSuccess) e = launch_collide(c, k, 1);
        k.zlo = k.nz - 1;
        k.zhi = k.nz;
        if (e == cudaSuccess) e = launch_collide(c, k, 1);
    } else {
        e = launch_collide(c, c->kp, has_solids(c));
    }
    if (c->f16) c->rs ^= 1;   // the slots are now relative to the densities the collide pass used
    return e;
}

cudaError_t record(lbm_ctx* c) {
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        c->ev.push_back(e);
    }
    return cudaEventRecord(c->ev[c->ev_used++], c->stream);
}

// Accumulates the event intervals recorded so far: events come as
// [e0 psi e1 collide e2] per step.
cudaError_t drain_timing(lbm_ctx* c) {
    if (c->ev_used == 0) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(c->ev[c->ev_used - 1]);
    if (e != cudaSuccess) return e;
    for (size_t k = 0; k + 2 < c->ev_used; k += 3) {
        float a = 0.f, b = 0.f;
        if ((e = cudaEventElapsedTime(&a, c->ev[k], c->ev[k + 1])) != cudaSuccess) return e;
        if ((e = cudaEventElapsedTime(&b, c->ev[k + 1], c->ev[k + 2])) != cudaSuccess) return e;
        c->ms[1] += a;   // collide runs first in a step
        c->ms[0] += b;
        c->launches[1] += 1;
        if ((c->kp.multiphase || c->f16) && !c->onepass) c->launches[0] += 1;
    }
    c->ev_used = 0;
    return cudaSuccess;
}

lbm_status read_status(lbm_ctx* c) {
    unsigned st = 0;
    CK(c, cudaMemcpyAsync(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->sticky == LBM_OK) {
        if (st & lbm::ST_TIMEOUT) {
            c->sticky = LBM_ERR_TIMEOUT;
            c->err = "a wait for populations staged by tensor copies ran out of time (the step was abandoned)";
        } else if (st & lbm::ST_UNSTABLE) {
            c->sticky = LBM_ERR_UNSTABLE;
            c->err = "non-finite or non-positive density on a fluid cell";
        } else if (st & lbm::ST_EOS_RANGE) {
            c->sticky = LBM_ERR_EOS_RANGE;
            c->err = "psi^2 < 0: density outside the range of the equation of state (psi clamped to 0)";
        }
    }
    return c->sticky;
}

// copy helper: device destination or host destination through the stream
// Host transfers go through one staging buffer, allocated on first use and grown on demand, so
// a context that is only fed from device memory holds no more than its resident state.
cudaError_t ensure_staging(lbm_ctx* c, size_t floats) {
    if (c->staging_floats >= floats) return cudaSuccess;
    if (c->staging) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        cudaFree(c->staging);
        c->bytes -= c->staging_floats * sizeof(float);
        c->staging = nullptr;
        c->staging_floats = 0;
    }
    cudaError_t e = cudaMalloc((void**)&c->staging, floats * sizeof(float));
    if (e != cudaSuccess) {
        c->staging = nullptr;
        return e;
    }
    c->staging_floats = floats;
    c->bytes += floats * sizeof(float);
    return cudaSuccess;
}

// Device bytes a context holds once initialised (host staging excluded).
size_t resident_bytes(const KParams& k, int Q, bool f16, bool with_solid, bool onepass) {
    const size_t n = (size_t)k.ncell;
    size_t b = (size_t)Q * (size_t)k.plane * (f16 ? 2 : sizeof(float)) * (onepass ? 2 : 1);   // populations
    if (f16) b += 2 * n * sizeof(float);                                   // two density fields
    b += n * sizeof(float);                                   // psi
    b += 64;                                                  // status word
    b += (size_t)lbm::moments_partial_blocks(k) * 4 * sizeof(double) + 4 * sizeof(double);
    if (with_solid) b += n * sizeof(uint32_t) + n;            // neighbour mask + solid copy
    return b;
}

lbm_status copy_out(lbm_ctx* c, void* dst, const void* src, size_t bytes, int on_device) {
    CK(c, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_params(lbm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->lattice = 19;
    p->nx = p->ny = p->nz = 32;
    p->eos = LBM_EOS_NONE;
    p->G = -1.0;
    p->sigma = 0.1;
    const double s[10] = {1.0, 1.0, 1.2, 0.6, 1.2, 0.6, 1.2, 1.2, 1.2, 1.2};
    for (int i = 0; i < 10; ++i) p->s[i] = s[i];
    p->psi_ext_rho = -1.0;
}

lbm_status lbm_create(const lbm_params* params, void* cuda_stream, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    lbm_status v = validate(params, why);
    if (v != LBM_OK) return fail(nullptr, v, why);
    lbm_ctx* c = new lbm_ctx();
    c->p = *params;
    c->Q = params->lattice;
    c->stream = (cudaStream_t)cuda_stream;
    const long long n = (long long)params->nx * params->ny * params->nz;
    const long long plane = (n + 63) / 64 * 64;   // 256-byte aligned planes
    c->kp = derive(*params, plane);
    c->partial_blocks = lbm::moments_partial_blocks(c->kp);
    auto alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) c->bytes += bytes;
        return e;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    c->f16 = params->store == LBM_STORE_FP16;
    set_layout(c, false);
    const size_t esize = c->f16 ? 2 : sizeof(float);   // FP16 slots are __half
    if (e == cudaSuccess) e = alloc((void**)&c->f, (size_t)c->Q * plane * esize);
    if (e == cudaSuccess)
        for (int i = 0; i < c->Q; ++i)
            c->kp.fq[i] = reinterpret_cast<float*>(reinterpret_cast<char*>(c->f) + (size_t)i * plane * esize);
    for (int k = 0; k < 2 && c->f16 && e == cudaSuccess; ++k) e = alloc((void**)&c->rbuf[k], (size_t)n * sizeof(float));
    c->onepass = params->onepass != 0;
    if (c->onepass && e == cudaSuccess) {
        e = alloc((void**)&c->f2, (size_t)c->Q * plane * sizeof(float));
        if (e == cudaSuccess)
            for (int i = 0; i < c->Q; ++i) c->kp.gq[i] = c->f2 + (size_t)i * plane;
    }
    if (params->onepass == 2 && e == cudaSuccess && !setup_staging(c)) e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = alloc((void**)&c->psi, (size_t)n * sizeof(float));
    if (e == cudaSuccess) e = alloc((void**)&c->status, 64);
    if (e == cudaSuccess) e = alloc((void**)&c->partials, (size_t)c->partial_blocks * 4 * sizeof(double));
    if (e == cudaSuccess) e = alloc((void**)&c->sums, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, 64, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->psi, 0, (size_t)n * sizeof(float), c->stream);
    if (e != cudaSuccess) {
        lbm_status s = e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
        std::string msg = std::string("device allocation failed: ") + cudaGetErrorString(e);
        (void)cudaGetLastError();
        lbm_destroy(c);
        return fail(nullptr, s, msg);
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx* c, const float* rho, const float* u, const uint8_t* solid, int on_device) {
    if (!c) return LBM_ERR_ARG;
    if (!rho || !u) return fail(c, LBM_ERR_ARG, "rho and u are required");
    const long long n = c->kp.ncell;
    const float* d_rho = rho;
    const float* d_u = u;
    if (!on_device) {
        CK(c, ensure_staging(c, 4 * (size_t)n));
        CK(c, cudaMemcpyAsync(c->staging, rho, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->staging + n, u, 3 * n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        d_rho = c->staging;
        d_u = c->staging + n;
    }
    if (solid && c->onepass) return fail(c, LBM_ERR_ARG, "onepass contexts take no solid mask");
    if (solid) {
        if (!c->nbmask) {
            CK(c, cudaMalloc((void**)&c->nbmask, n * sizeof(uint32_t)));
            c->bytes += n * sizeof(uint32_t);
        }
        if (!c->solid_dev) {
            CK(c, cudaMalloc((void**)&c->solid_dev, n));
            c->bytes += n;
        }
        CK(c, cudaMemcpyAsync(c->solid_dev, solid, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
        CK(c, lbm::launch_nbmask(c->kp, c->Q, c->solid_dev, c->nbmask, c->stream));
    } else if (c->nbmask) {
        // walls are handled arithmetically; no mask means "no interior solids"
        CK(c, cudaFree(c->nbmask));
        c->bytes -= n * sizeof(uint32_t);
        c->nbmask = nullptr;
    }
    c->tile_flags.clear();
    set_layout(c, solid != nullptr);
    if (c->onepass) {
        // natural-order populations into the other copy, then shifted into the pull layout
        lbm::KParams kn = c->kp;
        for (int i = 0; i < 27; ++i) kn.fq[i] = c->kp.gq[i];
        lbm::Bufs bn = bufs(c);
        bn.f = c->f2;
        CK(c, c->Q == 19 ? lbm::launch_init_q19(kn, bn, d_rho, d_u, c->stream)
                         : lbm::launch_init_q27(kn, bn, d_rho, d_u, c->stream));
        CK(c, c->Q == 19 ? lbm::launch_pull_store_q19(c->kp, c->f2, c->kp.plane, c->f, c->stream)
                         : lbm::launch_pull_store_q27(c->kp, c->f2, c->kp.plane, c->f, c->stream));
        c->parity = 2;
        c->t = 0;
        c->sticky = LBM_OK;
        CK(c, cudaMemsetAsync(c->status, 0, 64, c->stream));
        CK(c, run_psi(c));
        c->initialised = true;
        if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }
    CK(c, c->Q == 19 ? lbm::launch_init_q19(c->kp, bufs(c), d_rho, d_u, c->stream)
                     : lbm::launch_init_q27(c->kp, bufs(c), d_rho, d_u, c->stream));
    c->parity = 0;
    c->t = 0;
    c->sticky = LBM_OK;
    CK(c, cudaMemsetAsync(c->status, 0, 64, c->stream));
    CK(c, run_psi(c));
    c->initialised = true;
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int32_t n) {
    if (!c) return LBM_ERR_ARG;
    if (n < 0) return fail(c, LBM_ERR_ARG, "n must be >= 0");
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "lbm_step before lbm_init_fields");
    if (c->sticky != LBM_OK) return c->sticky;
    if (c->onepass) {
        for (int32_t k = 0; k < n; ++k) {
            if (c->timing) CK(c, record(c));
            CK(c, run_onepass(c));
            if (c->timing) CK(c, record(c));
            if (c->timing) CK(c, record(c));
            c->t += 1;
        }
        return LBM_OK;
    }
    if (has_solids(c) && !zwalls_only(c) && !c->timing && !c->f16 && n > 0 &&
        (unsigned long long)c->Q * (unsigned long long)c->kp.plane <= 0xFFFFFFFFull) {
        // walls or solids: the tile path, which runs solid-free tiles without solid handling
        if (!c->self_batch) {
            lbm_ctx* self[1] = {c};
            lbm_status bs = lbm_batch_create(self, 1, c->stream, &c->self_batch);
            if (bs != LBM_OK) return fail(c, bs, std::string("tile path: ") + lbm_last_error(nullptr));
        }
        lbm_status bs = lbm_batch_step(c->self_batch, n);
        if (bs != LBM_OK) return fail(c, bs, std::string("tile path: ") + lbm_batch_last_error(c->self_batch));
        return LBM_OK;
    }
    for (int32_t k = 0; k < n; ++k) {
        // psi of the current state is valid on entry: collide-stream, then density/psi of the new state
        if (c->timing) CK(c, record(c));
        CK(c, run_collide(c));
        c->parity ^= 1;
        if (c->timing) CK(c, record(c));
        CK(c, run_psi(c));
        if (c->timing) CK(c, record(c));
        c->t += 1;
    }
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    return read_status(c);
}

lbm_status lbm_get_moments(lbm_ctx* c, float* rho, float* u, double* sums, int on_device) {
    if (!c) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "lbm_get_moments before lbm_init_fields");
    const long long n = c->kp.ncell;
    if (!on_device && (rho || u)) CK(c, ensure_staging(c, 4 * (size_t)n));
    float* d_rho = on_device ? rho : (rho ? c->staging : nullptr);
    float* d_u = on_device ? u : (u ? c->staging + n : nullptr);
    int nb = 0;
    const int s = has_solids(c);
    if (c->onepass) CK(c, run_psi(c));   // the one-pass step keeps no psi field
    CK(c, c->Q == 19 ? lbm::launch_moments_q19(c->kp, c->parity, s, bufs(c), d_rho, d_u, c->partials, &nb, c->stream)
                     : lbm::launch_moments_q27(c->kp, c->parity, s, bufs(c), d_rho, d_u, c->partials, &nb, c->stream));
    CK(c, lbm::launch_finish_sums(c->partials, nb, c->sums, c->stream));
    if (!on_device) {
        if (rho) CK(c, cudaMemcpyAsync(rho, d_rho, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        if (u) CK(c, cudaMemcpyAsync(u, d_u, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    if (sums) CK(c, cudaMemcpyAsync(sums, c->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return read_status(c);
}

lbm_status lbm_get_psi(lbm_ctx* c, float* psi, int on_device) {
    if (!c || !psi) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "lbm_get_psi before lbm_init_fields");
    if (c->onepass) CK(c, run_psi(c));
    lbm_status s = copy_out(c, psi, c->psi, c->kp.ncell * sizeof(float), on_device);
    if (s != LBM_OK) return s;
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, float* f, int on_device) {
    if (!c || !f) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "lbm_get_populations before lbm_init_fields");
    const long long n = c->kp.ncell;
    if (!on_device) CK(c, ensure_staging(c, (size_t)c->Q * n));
    float* dst = on_device ? f : c->staging;
    const int s = has_solids(c);
    CK(c, c->Q == 19 ? lbm::launch_gather_q19(c->kp, c->parity, s, bufs(c), dst, c->stream)
                     : lbm::launch_gather_q27(c->kp, c->parity, s, bufs(c), dst, c->stream));
    if (!on_device) CK(c, cudaMemcpyAsync(f, dst, (size_t)c->Q * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const float* f, int on_device) {
    if (!c || !f) return LBM_ERR_ARG;
    const long long n = c->kp.ncell;
    if (c->onepass) {
        const float* d_f = f;
        if (!on_device) {
            CK(c, ensure_staging(c, (size_t)c->Q * n));
            CK(c, cudaMemcpyAsync(c->staging, f, (size_t)c->Q * n * sizeof(float), cudaMemcpyHostToDevice,
                                  c->stream));
            d_f = c->staging;
        }
        CK(c, c->Q == 19 ? lbm::launch_pull_store_q19(c->kp, d_f, n, c->f, c->stream)
                         : lbm::launch_pull_store_q27(c->kp, d_f, n, c->f, c->stream));
        c->parity = 2;
        c->sticky = LBM_OK;
        CK(c, cudaMemsetAsync(c->status, 0, 64, c->stream));
        CK(c, run_psi(c));
        c->initialised = true;
        CK(c, cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }
    if (c->f16) {
        // densities of the given state, then the slots relative to them
        const float* d_f = f;
        if (!on_device) {
            CK(c, ensure_staging(c, (size_t)c->Q * n));
            CK(c, cudaMemcpyAsync(c->staging, f, (size_t)c->Q * n * sizeof(float), cudaMemcpyHostToDevice,
                                  c->stream));
            d_f = c->staging;
        }
        CK(c, c->Q == 19 ? lbm::launch_f16_restore_q19(c->kp, bufs(c), d_f, c->stream)
                         : lbm::launch_f16_restore_q27(c->kp, bufs(c), d_f, c->stream));
    } else {
        CK(c, cudaMemcpy2DAsync(c->f, c->kp.plane * sizeof(float), f, n * sizeof(float), n * sizeof(float), c->Q,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    }
    c->parity = 0;
    c->sticky = LBM_OK;
    CK(c, cudaMemsetAsync(c->status, 0, 64, c->stream));
    CK(c, run_psi(c));
    c->initialised = true;
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx* c, void* cuda_stream) {
    if (!c) return LBM_ERR_ARG;
    if (c->self_batch) {   // bound to the old stream
        lbm_batch_destroy(c->self_batch);
        c->self_batch = nullptr;
    }
    c->stream = (cudaStream_t)cuda_stream;
    return LBM_OK;
}

lbm_status lbm_set_kernel_timing(lbm_ctx* c, int enable) {
    if (!c) return LBM_ERR_ARG;
    CK(c, drain_timing(c));
    c->timing = enable != 0;
    c->ms[0] = c->ms[1] = 0.0;
    c->launches[0] = c->launches[1] = 0;
    return LBM_OK;
}

lbm_status lbm_get_kernel_timing(lbm_ctx* c, double ms[2], int64_t launches[2]) {
    if (!c) return LBM_ERR_ARG;
    CK(c, drain_timing(c));
    if (ms) { ms[0] = c->ms[0]; ms[1] = c->ms[1]; }
    if (launches) { launches[0] = c->launches[0]; launches[1] = c->launches[1]; }
    return LBM_OK;
}

int64_t lbm_step_count(const lbm_ctx* c) { return c ? c->t : -1; }

size_t lbm_device_bytes(const lbm_ctx* c) { return c ? c->bytes : 0; }

lbm_status lbm_estimate_bytes(const lbm_params* params, int32_t with_solid, size_t* bytes) {
    if (!bytes) return fail(nullptr, LBM_ERR_ARG, "bytes is NULL");
    *bytes = 0;
    std::string why;
    lbm_status v = validate(params, why);
    if (v != LBM_OK) return fail(nullptr, v, why);
    const long long n = (long long)params->nx * params->ny * params->nz;
    const KParams k = derive(*params, (n + 63) / 64 * 64);
    *bytes = resident_bytes(k, params->lattice, params->store == LBM_STORE_FP16, with_solid != 0,
                            params->onepass != 0);
    return LBM_OK;
}

lbm_status lbm_contact(lbm_ctx* c, float rho_threshold, int32_t* out, int on_device) {
    if (!c || !out) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "lbm_contact before lbm_init_fields");
    if (!std::isfinite(rho_threshold)) return fail(c, LBM_ERR_ARG, "rho_threshold must be finite");
    int* d_out = on_device ? reinterpret_cast<int*>(out) : reinterpret_cast<int*>(c->sums);   // sums: 32 bytes
    CK(c, lbm::launch_contact_init(d_out, c->stream));
    if (has_solids(c))
        CK(c, c->Q == 19 ? lbm::launch_contact_q19(c->kp, c->parity, bufs(c), rho_threshold, d_out, c->stream)
                         : lbm::launch_contact_q27(c->kp, c->parity, bufs(c), rho_threshold, d_out, c->stream));
    if (on_device) return LBM_OK;
    int32_t h[6];
    CK(c, cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::memcpy(out, h, sizeof(h));
    return read_status(c);
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->self_batch) lbm_batch_destroy(c->self_batch);
    if (c->stream || c->f) (void)cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->ev) (void)cudaEventDestroy(e);
    void* ptrs[] = {c->f, c->psi, c->nbmask, c->status, c->partials, c->sums, c->staging, c->solid_dev,
                    c->rbuf[0], c->rbuf[1], c->f2};
    for (void* p : ptrs)
        if (p) (void)cudaFree(p);
    delete c;
}

const char* lbm_last_error(const lbm_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

lbm_status lbm_debug_stage_timeout(lbm_ctx* c, int32_t enable) {
    if (!c) return LBM_ERR_ARG;
    if (!c->staged) return fail(c, LBM_ERR_STATE, "this context does not stage populations with tensor copies");
    c->stage_timeout_test = enable != 0;
    return LBM_OK;
}

int32_t lbm_staged_copies(const lbm_ctx* c) { return c ? c->staged : 0; }

uint64_t lbm_debug_bounds_violations(void) {
    return lbm::bounds_violations_q19() + lbm::bounds_violations_q27();
}

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "LBM_OK";
        case LBM_ERR_ARG: return "LBM_ERR_ARG";
        case LBM_ERR_OOM: return "LBM_ERR_OOM";
        case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
        case LBM_ERR_UNSTABLE: return "LBM_ERR_UNSTABLE";
        case LBM_ERR_EOS_RANGE: return "LBM_ERR_EOS_RANGE";
        case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
        case LBM_ERR_STATE: return "LBM_ERR_STATE";
    }
    return "LBM_UNKNOWN";
}

}  // extern "C"

// ------------------------------------------------------------------ lattice-independent kernels
namespace lbm {
namespace {

__host__ __device__ constexpr int ex27(int i) {
    constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int ey27(int i) {
    constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int ez27(int i) {
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    return t[i];
}

__global__ void contact_init_kernel(int* out) {
    const int t = threadIdx.x;
    if (t < 6) out[t] = t < 2 ? 0 : ((t & 1) ? INT_MIN : INT_MAX);
}

// bit i of nbmask[x] <=> x + e_i is an interior solid cell (bit 0: x itself).  Walls are not
// stored here; the kernels add them from the position.
__global__ void nbmask_kernel(KParams kp, int Q, const uint8_t* __restrict__ solid, uint32_t* __restrict__ out) {
    const long long n = kp.ncell;
    const long long nxy = (long long)kp.nx * kp.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % kp.nx), y = (int)((idx / kp.nx) % kp.ny), z = (int)(idx / nxy);
        uint32_t bits = 0u;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            if (i >= Q) break;
            int xx = x + ex27(i), yy = y + ey27(i), zz = z + ez27(i);
            bool outside = false;
            if (xx < 0 || xx >= kp.nx) { if (kp.wall_x) outside = true; else xx = (xx + kp.nx) % kp.nx; }
            if (yy < 0 || yy >= kp.ny) { if (kp.wall_y) outside = true; else yy = (yy + kp.ny) % kp.ny; }
            if (zz < 0 || zz >= kp.nz) { if (kp.wall_z) outside = true; else zz = (zz + kp.nz) % kp.nz; }
            if (!outside && solid[zz * nxy + (long long)yy * kp.nx + xx]) bits |= 1u << i;
        }
        out[idx] = bits;
    }
}

// Sums per-block partials in a fixed order (one block, fixed thread assignment, fixed tree).
__global__ void finish_sums_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ sums) {
    __shared__ double red[4][256];
    const int t = threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = t; b < nblocks; b += 256)
        for (int k = 0; k < 4; ++k) acc[k] += partials[4 * (long long)b + k];
    for (int k = 0; k < 4; ++k) red[k][t] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < 4; ++k) red[k][t] += red[k][t + w];
        __syncthreads();
    }
    if (t < 4) sums[t] = red[t][0];
}

}  // namespace

cudaError_t launch_nbmask(const KParams& kp, int Q, const uint8_t* solid, uint32_t* nbmask, cudaStream_t st) {
    const long long blocks = (kp.ncell + 255) / 256;
    nbmask_kernel<<<(int)(blocks < 152LL * 64 ? blocks : 152LL * 64), 256, 0, st>>>(kp, Q, solid, nbmask);
    return cudaGetLastError();
}

cudaError_t launch_finish_sums(const double* partials, int nblocks, double* sums, cudaStream_t st) {
    finish_sums_kernel<<<1, 256, 0, st>>>(partials, nblocks, sums);
    return cudaGetLastError();
}

cudaError_t launch_contact_init(int* out, cudaStream_t st) {
    contact_init_kernel<<<1, 32, 0, st>>>(out);
    return cudaGetLastError();
}

void set_thread_error(const char* msg) { g_create_error = msg; }

long long moments_partial_blocks(const KParams& kp) {
    // matches the collide/moments launch shape (32 x 4 x 2 cells per block)
    return (long long)((kp.nx + 31) / 32) * ((kp.ny + 3) / 4) * ((kp.nz + 1) / 2);
}

}  // namespace lbm
