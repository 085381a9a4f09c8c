// Internal layout of an lbm_ctx, shared by the C ABI (capi.cu) and the multi-domain batch
// (batch.cu).  Not part of the public interface.
#pragma once

#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

struct lbm_ctx {
    lbm_params p{};
    int Q = 19;
    lbm::KParams kp{};
    cudaStream_t stream = nullptr;
    int device = 0;
    // device state
    float* f = nullptr;          // Q planes of `plane` slots (AA layout): floats, or __half with f16
    int f16 = 0;                 // shifted FP16 store (LBM_STORE_FP16)
    int paired = 0;              // f16 slots in the x-paired layout (see KParams::paired)
    int onepass = 0;             // one-pass layout: f is the copy being read, f2 the one written
    float* f2 = nullptr;
    // one-pass contexts with full 32 x 4 tiles stage each plane's populations with tensor copies:
    // one tensor map per population copy (tmap_base[k] is the copy tmap[k] describes)
    int staged = 0;
    CUtensorMap tmap[2];
    const void* tmap_base[2] = {nullptr, nullptr};
    int stage_timeout_test = 0;  // lbm_debug_stage_timeout
    float* rbuf[2] = {nullptr, nullptr};   // f16: density fields, see bufs() in capi.cu
    int rs = 0;
    float* psi = nullptr;        // ncell floats
    uint32_t* nbmask = nullptr;  // ncell words, only when a solid mask was given
    unsigned* status = nullptr;  // device status word
    double* partials = nullptr;  // moments partial sums (4 per block)
    double* sums = nullptr;      // 4 doubles
    float* staging = nullptr;    // host-transfer buffer, allocated on first use
    size_t staging_floats = 0;
    uint8_t* solid_dev = nullptr;
    size_t bytes = 0;
    // per 32 x 4 column and z plane: 1 if some cell there has a solid neighbour (mask only),
    // computed on first use by a multi-domain batch, cleared when the fields are re-initialised
    std::vector<uint8_t> tile_flags;
    int tile_flags_tw = 0, tile_flags_th = 0;   // the column shape tile_flags was computed for
    // domains with walls or solids step through a one-member batch (created on first use): its
    // tiles away from solids take the kernels without solid handling
    lbm_batch* self_batch = nullptr;
    long long partial_blocks = 0;
    // host state
    int parity = 0;              // 0: natural layout, 1: swapped (after an odd number of AA steps)
    long long t = 0;
    bool initialised = false;
    lbm_status sticky = LBM_OK;
    std::string err;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double ms[2] = {0.0, 0.0};
    long long launches[2] = {0, 0};
};

