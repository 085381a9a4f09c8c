// Multi-domain batch (lbm_batch_*): many independent domains advanced together.
//
// Members are grouped by (lattice, solid handling, physical parameters).  Per time step each group
// costs one collide-stream launch and one density/psi launch whose blocks are tiles of every
// member of the group (up to 64 members per launch), instead of two launches per domain.  The
// group's physical parameters (rates, equation of state, forces) and the launch's member table
// (geometry and buffer addresses, 64 bytes a member) are passed by value in the kernel
// parameters, so a block reads them from the constant bank as the single-domain kernel does.
// The per-cell arithmetic is the single-domain code, so a member's result is bitwise the same
// as stepping it alone.  Whole runs are replayed from a CUDA graph: a WHILE
// conditional node repeats a two-step body until a device-side counter runs out, so n steps are
// one graph launch; where conditional nodes are unavailable the two-step graph is launched n/2
// times.  lbm_batch_tune times the candidate z-chunks per group on the live state.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "ctx_internal.h"
#include "lbm_internal.h"

using lbm::BatchDom;
using lbm::BatchDomTable;
using lbm::BatchRun;
using lbm::div_magic;
using lbm::BatchTile;
using lbm::KParams;

namespace {

// One launch of a group: up to BATCH_LAUNCH_DOMS members and their tile ranges in the group's
// tile arrays.
struct Launch {
    BatchDomTable tab{};
    int t0 = 0, nt = 0;             // collide tiles
    int p0 = 0, np = 0;             // density/psi tiles (the collide tiles in a solid-handling group)
    int r0 = 0, nr = 0;             // density/psi runs of whole planes (plain groups)
};

struct Group {
    int Q = 19, solids = 0;
    KParams phys{};                 // physical parameters shared by the members (geometry zeroed)
    std::vector<int> members;       // members with tiles in this group
    int zchunk = 0;                 // 0 = automatic
    int shape = 0;                  // tile shape: index into lbm::BATCH_SHAPES
    std::vector<Launch> launches;
    BatchTile* tiles = nullptr;     // collide tiles, then density/psi tiles (device)
    int ntiles = 0;                 // collide tiles
    BatchRun* runs = nullptr;       // density/psi runs (device)
};

__global__ void set_counter_kernel(int* counter, int value) { *counter = value; }

// Last node of the loop body: one more two-step iteration done; stop when the count runs out.
__global__ void loop_tick_kernel(cudaGraphConditionalHandle h, int* counter) {
    if (--(*counter) <= 0) cudaGraphSetConditional(h, 0);
}

bool has_solid_work(const lbm_ctx* c) { return c->nbmask != nullptr || c->kp.wall_x || c->kp.wall_y || c->kp.wall_z; }

// The physical part of a member's parameters: geometry, addresses and tiling fields zeroed, so
// that members with equal physics compare equal byte for byte.
KParams physics_of(const KParams& k) {
    KParams p;
    std::memcpy(&p, &k, sizeof(KParams));
    p.nx = p.ny = p.nz = 0;
    p.wall_x = p.wall_y = p.wall_z = 0;
    p.plane = p.ncell = 0;
    for (float*& q : p.fq) q = nullptr;
    for (float*& q : p.gq) q = nullptr;
    p.zchunk = 0;
    p.zlo = p.zhi = 0;
    p.paired = p.hx = 0;        // storage layout (FP16 only), not physics
    return p;
}

BatchDom dom_of(const lbm_ctx* c) {
    BatchDom d{};
    d.nx = c->kp.nx;
    d.ny = c->kp.ny;
    d.nz = c->kp.nz;
    d.wall_x = c->kp.wall_x;
    d.wall_y = c->kp.wall_y;
    d.wall_z = c->kp.wall_z;
    d.plane = c->kp.plane;
    d.base = c->kp.fq[0];
    d.psi = c->psi;
    d.nbmask = c->nbmask;
    d.status = c->status;
    div_magic((uint32_t)c->kp.nx, d.mx, d.sx);
    div_magic((uint32_t)c->kp.ny, d.my, d.sy);
    return d;
}

}  // namespace

struct lbm_batch {
    std::vector<lbm_ctx*> members;
    std::vector<KParams> seen;      // member parameters the groups were built from
    std::vector<BatchDom> table;    // member geometry and addresses the groups were built from
    std::vector<Group> groups;
    cudaStream_t stream = nullptr;
    int* counter = nullptr;         // loop counter of the graph (device)
    cudaStream_t cap = nullptr;     // capture stream
    cudaGraphExec_t exec = nullptr;
    int graph_parity = -1;          // AA phase the graph was recorded for
    int graph_mode = 0;             // 0 none yet, 1 WHILE conditional node, 2 replayed two-step graph
    std::vector<cudaStream_t> side; // one per group: the groups of a pass run concurrently
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> done;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& m) {
    if (b) b->err = m;
    else lbm::set_thread_error(m.c_str());
    return s;
}

#define BCK(b, call)                                                                                 \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,            \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

void free_tiles(Group& g) {
    if (g.tiles) cudaFree(g.tiles);
    if (g.runs) cudaFree(g.runs);
    g.tiles = nullptr;
    g.runs = nullptr;
    g.ntiles = 0;
    g.launches.clear();
}

void drop_graph(lbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_parity = -1;
    b->graph_mode = 0;
}

constexpr int ZC_WHOLE = 1 << 30;   // a z-chunk candidate: every column marches through all its planes
constexpr int ZC_AUTO_MAX = 32;   // automatic z-chunks: longer marches gain little, and in a mix of
                                  // uneven members shorter blocks balance the last wave

// flags[(z * nyb + yb) * nxb + xb] = 1 if a cell of the blockDim.x x blockDim.y column (xb, yb) in
// plane z has a solid neighbour or is solid (its neighbour mask is nonzero).
__global__ void tile_flags_kernel(const uint32_t* __restrict__ nbmask, int nx, int ny, uint8_t* flags) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    bool any = false;
    if (x < nx && y < ny) any = nbmask[((long long)z * ny + y) * nx + x] != 0u;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        flags[((long long)z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = any ? 1 : 0;
}

// Mask flags of a member for tw x th columns (cached on the context until its fields are
// re-initialised or another tile shape asks).
lbm_status member_tile_flags(lbm_batch* b, lbm_ctx* c, int tw, int th) {
    const KParams& k = c->kp;
    const long long nxb = (k.nx + tw - 1) / tw, nyb = (k.ny + th - 1) / th;
    const size_t n = (size_t)(nxb * nyb * k.nz);
    if (!c->nbmask || (c->tile_flags.size() == n && c->tile_flags_tw == tw && c->tile_flags_th == th)) return LBM_OK;
    uint8_t* d = nullptr;
    BCK(b, cudaMalloc((void**)&d, n));
    c->tile_flags.assign(n, 1);
    c->tile_flags_tw = tw;
    c->tile_flags_th = th;
    tile_flags_kernel<<<dim3((unsigned)nxb, (unsigned)nyb, (unsigned)k.nz), dim3(tw, th), 0, b->stream>>>(
        c->nbmask, k.nx, k.ny, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->tile_flags.data(), d, n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d);
    if (e != cudaSuccess) {
        c->tile_flags.clear();
        return bfail(b, LBM_ERR_CUDA, std::string("tile flags: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

// Tiles of the members of a group: tw x th cells in (x, y) (the group's shape) and a run of z planes.  Along every
// column the planes are split into runs that need solid handling (a cell with a solid neighbour:
// mask, or the first / last plane, row or column next to a wall) and runs that do not; runs are
// cut into chunks of at most zc planes, chosen so that the whole group gives a few waves of
// resident blocks (or the group's fixed zchunk).  A member with solids contributes its solid-free
// chunks to the group without solid handling and the others to the solid group of its physics,
// so only cells near solids pay for the solid tests.
//
// Where a row leaves 1 .. 16 cells past its last full tile width (tw = 32), those cells form narrow
// columns, 16 cells wide and twice as high, which the same blocks step (BatchTile::narrow): a
// 32-wide tile there would leave 16 to 31 of its 32 lanes per row idle.
//
// The density/psi pass of a group without solid handling covers the planes in which no column needs
// it (every plane of a member without solids) as runs of RUN_CELLS consecutive cells, and only the
// solid-free columns of the other planes as tiles: the pass needs no stencil, so nothing ties its
// threads to rows, and rows that do not fill a tile's width leave no lanes idle.
#ifndef LBM_BATCH_RUNS
#define LBM_BATCH_RUNS 1
#endif
#ifndef LBM_BATCH_NARROW
#define LBM_BATCH_NARROW 1
#endif
#ifndef LBM_BATCH_LPT
#define LBM_BATCH_LPT 1
#endif
constexpr uint32_t RUN_CELLS = 2048;

struct Column {
    int x0, y0, w, h, narrow;
};

// the columns of a member for tiles tw x th: full-width columns, then the narrow ones (if any)
std::vector<Column> member_columns(const KParams& k, int tw, int th) {
    std::vector<Column> cols;
    const int r = k.nx % tw;
    const bool narrow = LBM_BATCH_NARROW && tw > lbm::BATCH_NARROW_BX && r > 0 && r <= lbm::BATCH_NARROW_BX;
    const int wmain = narrow ? k.nx - r : k.nx;
    for (int y0 = 0; y0 < k.ny; y0 += th)
        for (int x0 = 0; x0 < wmain; x0 += tw) cols.push_back({x0, y0, tw, th, 0});
    if (narrow) {
        const int hn = tw * th / lbm::BATCH_NARROW_BX;
        for (int y0 = 0; y0 < k.ny; y0 += hn) cols.push_back({wmain, y0, lbm::BATCH_NARROW_BX, hn, 1});
    }
    return cols;
}

lbm_status build_tiles(lbm_batch* b, Group& g) {
    free_tiles(g);
    if (g.shape < 0 || g.shape >= lbm::BATCH_NSHAPES) return bfail(b, LBM_ERR_ARG, "unknown tile shape");
    const lbm::BatchShape& sh = lbm::BATCH_SHAPES[g.shape];
    const int tw = sh.bx, th = sh.by;
    const int fw = lbm::BATCH_NARROW_BX, fh = th;   // mask flags grid: both column kinds are unions of its cells
    const int resident = g.Q == 19 ? sh.minb19 : sh.minb27;
    const bool use_runs = LBM_BATCH_RUNS && !g.solids;
    long long ncols = 0;
    for (int d : g.members) ncols += (long long)member_columns(b->members[d]->kp, tw, th).size();
    const long long target = 152LL * resident * 4;
    const long long chunks_auto = std::max(1LL, (target + ncols - 1) / std::max(ncols, 1LL));
    std::vector<BatchTile> t, pt;   // collide tiles; density/psi tiles
    std::vector<BatchRun> runs;
    std::vector<uint8_t> need;      // per plane of one column: needs solid handling
    std::vector<uint8_t> mixed;     // per plane: some column needs solid handling
    for (size_t j = 0; j < g.members.size(); ++j) {
        const int d = (int)(j % lbm::BATCH_LAUNCH_DOMS);   // slot in the launch's member table
        if (d == 0) {
            g.launches.emplace_back();
            g.launches.back().t0 = (int)t.size();
            g.launches.back().p0 = (int)pt.size();
            g.launches.back().r0 = (int)runs.size();
        }
        Launch& L = g.launches.back();
        L.tab.d[d] = b->table[g.members[j]];
        lbm_ctx* c = b->members[g.members[j]];
        const KParams& k = c->kp;
        const bool solid_work = has_solid_work(c);
        lbm_status fs = member_tile_flags(b, c, fw, fh);
        if (fs != LBM_OK) return fs;
        int zc;
        if (g.zchunk > 0) zc = std::min(g.zchunk, k.nz);            // the batch's tuned choice
        else if (k.zchunk > 0) zc = std::min(k.zchunk, k.nz);       // the member's own setting
        else {
            const long long ch = std::min<long long>(chunks_auto, k.nz);
            zc = std::min(ZC_AUTO_MAX, (int)((k.nz + ch - 1) / ch));
        }
        const int nxf = (k.nx + fw - 1) / fw, nyf = (k.ny + fh - 1) / fh;
        const std::vector<Column> cols = member_columns(k, tw, th);
        auto column_needs = [&](const Column& col) {
            const bool side = (k.wall_x && (col.x0 == 0 || col.x0 + col.w >= k.nx)) ||
                              (k.wall_y && (col.y0 == 0 || col.y0 + col.h >= k.ny));
            const int fx0 = col.x0 / fw, fx1 = std::min(nxf, (col.x0 + col.w + fw - 1) / fw);
            const int fy0 = col.y0 / fh, fy1 = std::min(nyf, (col.y0 + col.h + fh - 1) / fh);
            for (int z = 0; z < k.nz; ++z) {
                bool s2 = side || (k.wall_z && (z == 0 || z == k.nz - 1));
                if (c->nbmask)
                    for (int fy = fy0; fy < fy1 && !s2; ++fy)
                        for (int fx = fx0; fx < fx1 && !s2; ++fx)
                            s2 = c->tile_flags[((size_t)z * nyf + fy) * nxf + fx] != 0;
                need[z] = s2 ? 1 : 0;
            }
        };
        need.resize(k.nz);
        mixed.assign(k.nz, 0);
        if (solid_work)
            for (const Column& col : cols) {
                column_needs(col);
                for (int z = 0; z < k.nz; ++z) mixed[z] |= need[z];
            }
        const int member_t0 = (int)t.size() - L.t0, member_p0 = (int)pt.size() - L.p0;
        for (const Column& col : cols) {
            column_needs(col);
            for (int z0 = 0; z0 < k.nz;) {
                int z1 = z0 + 1;
                while (z1 < k.nz && need[z1] == need[z0] && z1 - z0 < zc) ++z1;
                const bool mine = solid_work ? (need[z0] != 0) == (g.solids != 0) : true;
                if (mine) t.push_back({d, col.x0, col.y0, z0, z1 - z0, col.narrow});
                z0 = z1;
            }
            if (use_runs)   // density/psi tiles: this column's solid-free planes among the mixed ones
                for (int z0 = 0; z0 < k.nz;) {
                    if (need[z0] || !mixed[z0]) {
                        ++z0;
                        continue;
                    }
                    int z1 = z0 + 1;
                    while (z1 < k.nz && !need[z1] && mixed[z1] && z1 - z0 < zc) ++z1;
                    pt.push_back({d, col.x0, col.y0, z0, z1 - z0, col.narrow});
                    z0 = z1;
                }
        }
        // z-chunk-major order within the member (as the single-domain grid): blocks resident at
        // the same time work on neighbouring columns of the same planes
        auto zmajor = [](const BatchTile& a, const BatchTile& b2) {
            return a.z0 != b2.z0 ? a.z0 < b2.z0 : (a.y0 != b2.y0 ? a.y0 < b2.y0 : a.x0 < b2.x0);
        };
        std::stable_sort(t.begin() + L.t0 + member_t0, t.end(), zmajor);
        std::stable_sort(pt.begin() + L.p0 + member_p0, pt.end(), zmajor);
        if (use_runs) {
            const uint32_t nxy = (uint32_t)k.nx * (uint32_t)k.ny;
            for (int z0 = 0; z0 < k.nz;) {
                if (mixed[z0]) {
                    ++z0;
                    continue;
                }
                int z1 = z0 + 1;
                while (z1 < k.nz && !mixed[z1]) ++z1;
                const uint32_t end = (uint32_t)z1 * nxy;
                for (uint32_t a = (uint32_t)z0 * nxy; a < end; a += std::min(RUN_CELLS, end - a))
                    runs.push_back({d, a, a + std::min(RUN_CELLS, end - a)});
                z0 = z1;
            }
        }
        L.nt = (int)t.size() - L.t0;
        L.np = (int)pt.size() - L.p0;
        L.nr = (int)runs.size() - L.r0;
    }
    // longest marches first within a launch: blocks start roughly in index order, so the short ones
    // fill the last wave instead of a few long ones running on alone
    if (LBM_BATCH_LPT)
        for (const Launch& L : g.launches)
            std::stable_sort(t.begin() + L.t0, t.begin() + L.t0 + L.nt,
                             [](const BatchTile& a, const BatchTile& b2) { return a.zc > b2.zc; });
    if (!use_runs)
        for (Launch& L : g.launches) {   // the density/psi pass runs over the collide tiles
            L.p0 = L.t0;
            L.np = L.nt;
        }
    else
        for (Launch& L : g.launches) L.p0 += (int)t.size();
    if (t.size() + pt.size() > 0x7fffffff || runs.size() > 0x7fffffff) return bfail(b, LBM_ERR_ARG, "too many tiles");
    const size_t nt = t.size() + pt.size();
    if (nt > 0) {
        t.insert(t.end(), pt.begin(), pt.end());
        BCK(b, cudaMalloc((void**)&g.tiles, nt * sizeof(BatchTile)));
        BCK(b, cudaMemcpyAsync(g.tiles, t.data(), nt * sizeof(BatchTile), cudaMemcpyHostToDevice, b->stream));
    }
    if (!runs.empty()) {
        BCK(b, cudaMalloc((void**)&g.runs, runs.size() * sizeof(BatchRun)));
        BCK(b, cudaMemcpyAsync(g.runs, runs.data(), runs.size() * sizeof(BatchRun), cudaMemcpyHostToDevice, b->stream));
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    g.ntiles = (int)(nt - pt.size());
    return LBM_OK;
}

// One collide launch of group g at AA phase `parity` (optionally bracketed by events).
cudaError_t collide_group(const Group& g, int parity, cudaStream_t st) {
    for (const Launch& L : g.launches) {
        const BatchTile* t = g.tiles + L.t0;
        cudaError_t e = g.Q == 19 ? lbm::launch_collide_batch_q19(g.phys, L.tab, t, L.nt, parity, g.solids, g.shape, st)
                                  : lbm::launch_collide_batch_q27(g.phys, L.tab, t, L.nt, parity, g.solids, g.shape, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t psi_group(const Group& g, int parity, cudaStream_t st) {
    if (!g.phys.multiphase) return cudaSuccess;
    for (const Launch& L : g.launches) {
        const BatchTile* t = g.tiles + L.p0;
        cudaError_t e = g.Q == 19 ? lbm::launch_psi_batch_q19(g.phys, L.tab, t, L.np, parity, g.solids, g.shape, st)
                                  : lbm::launch_psi_batch_q27(g.phys, L.tab, t, L.np, parity, g.solids, g.shape, st);
        if (e == cudaSuccess && L.nr > 0)
            e = g.Q == 19 ? lbm::launch_psi_runs_q19(g.phys, L.tab, g.runs + L.r0, L.nr, parity, st)
                          : lbm::launch_psi_runs_q27(g.phys, L.tab, g.runs + L.r0, L.nr, parity, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// (Re)build the groups, their member tables and tiles from the members' current parameters.  Walls-only members join both the plain group (interior tiles) and the
// solid-handling group (boundary tiles) of their physics.
lbm_status regroup(lbm_batch* b) {
    drop_graph(b);
    for (Group& g : b->groups) free_tiles(g);
    b->groups.clear();
    const int n = (int)b->members.size();
    b->seen.resize(n);
    b->table.resize(n);
    auto group_of = [&](int Q, int solids, const KParams& phys) -> Group& {
        for (Group& g : b->groups)
            if (g.Q == Q && g.solids == solids && std::memcmp(&g.phys, &phys, sizeof(KParams)) == 0) return g;
        Group g;
        g.Q = Q;
        g.solids = solids;
        g.phys = phys;
        b->groups.push_back(g);
        return b->groups.back();
    };
    for (int i = 0; i < n; ++i) {
        const lbm_ctx* c = b->members[i];
        if ((unsigned long long)c->Q * (unsigned long long)c->kp.plane > 0xFFFFFFFFull)
            return bfail(b, LBM_ERR_ARG, "a batch member holds 2^32 or more population values "
                                         "(Q x cells rounded up to 64); step it alone");
        std::memcpy(&b->seen[i], &c->kp, sizeof(KParams));
        b->table[i] = dom_of(c);
        const KParams phys = physics_of(c->kp);
        group_of(c->Q, 0, phys).members.push_back(i);   // solid-free tiles
        if (has_solid_work(c)) group_of(c->Q, 1, phys).members.push_back(i);
    }
    for (Group& g : b->groups) {
        lbm_status s = build_tiles(b, g);
        if (s != LBM_OK) return s;
    }
    return LBM_OK;
}

// Has any member changed (re-initialised with another solid mask) since the groups were built?
bool members_changed(const lbm_batch* b) {
    for (size_t i = 0; i < b->members.size(); ++i) {
        const BatchDom d = dom_of(b->members[i]);
        if (std::memcmp(&b->seen[i], &b->members[i]->kp, sizeof(KParams)) != 0 ||
            std::memcmp(&b->table[i], &d, sizeof(BatchDom)) != 0)
            return true;
    }
    return false;
}

// One pass (collide-stream or density/psi) of every group.  The groups' launches are
// independent within a pass -- tiles of one member in two groups touch disjoint cells, and the
// in-place AA update of a cell reads and writes only that cell's slots -- so they are forked onto
// one side stream each and joined before the next pass (in a captured graph: parallel nodes
// between two joins).  The next pass needs all of them: psi reads populations that neighbouring
// tiles wrote, and collide reads the psi halo.
cudaError_t pass(lbm_batch* b, bool collide, int parity, cudaStream_t st) {
    const size_t G = b->groups.size();
    if (G == 1) return collide ? collide_group(b->groups[0], parity, st) : psi_group(b->groups[0], parity, st);
    cudaError_t e = cudaSuccess;
    if (!b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    while (e == cudaSuccess && b->side.size() < G) {
        cudaStream_t s2 = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            b->side.push_back(s2);
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->done.push_back(ev);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, st);
    for (size_t k = 0; k < G && e == cudaSuccess; ++k) {
        e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
        if (e == cudaSuccess)
            e = collide ? collide_group(b->groups[k], parity, b->side[k]) : psi_group(b->groups[k], parity, b->side[k]);
        if (e == cudaSuccess) e = cudaEventRecord(b->done[k], b->side[k]);
    }
    for (size_t k = 0; k < G && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(st, b->done[k], 0);
    return e;
}

// One step of every member, starting at AA phase `parity` (psi of the current state valid).
cudaError_t step_once(lbm_batch* b, int parity, cudaStream_t st) {
    cudaError_t e = pass(b, true, parity, st);
    return e == cudaSuccess ? pass(b, false, parity ^ 1, st) : e;
}

lbm_status record_graph(lbm_batch* b, int parity) {
    drop_graph(b);
    if (!b->cap) BCK(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    // first choice: one WHILE node whose body is two steps and a counter tick
    cudaGraph_t g = nullptr;
    BCK(b, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    bool ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            cudaError_t e1 = step_once(b, parity, b->cap);
            cudaError_t e2 = e1 == cudaSuccess ? step_once(b, parity ^ 1, b->cap) : e1;
            if (e2 == cudaSuccess) {
                loop_tick_kernel<<<1, 1, 0, b->cap>>>(h, b->counter);
                e2 = cudaGetLastError();
            }
            cudaGraph_t out = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(b->cap, &out);
            ok = e2 == cudaSuccess && e3 == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (ok) {
        b->graph_mode = 1;
        b->graph_parity = parity;
        return LBM_OK;
    }
    (void)cudaGetLastError();
    b->exec = nullptr;
    // fallback: a plain two-step graph, replayed
    BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = step_once(b, parity, b->cap);
    cudaError_t e2 = e1 == cudaSuccess ? step_once(b, parity ^ 1, b->cap) : e1;
    cudaGraph_t g2 = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(b->cap, &g2);
    if (e2 != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e2));
    if (e3 != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e3));
    cudaError_t e4 = cudaGraphInstantiate(&b->exec, g2, 0);
    cudaGraphDestroy(g2);
    if (e4 != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e4));
    b->graph_mode = 2;
    b->graph_parity = parity;
    return LBM_OK;
}

void advance_members(lbm_batch* b, int n) {
    for (lbm_ctx* c : b->members) {
        c->t += n;
        c->parity ^= (n & 1);
    }
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int32_t n, void* cuda_stream, lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return bfail(nullptr, LBM_ERR_ARG, "a batch needs at least one context");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return bfail(nullptr, LBM_ERR_ARG, "NULL context in the batch");
        if (!ctxs[i]->initialised) return bfail(nullptr, LBM_ERR_STATE, "every context must be initialised");
        if (ctxs[i]->f16)
            return bfail(nullptr, LBM_ERR_ARG, "contexts with the FP16 store cannot join a batch");
        if (ctxs[i]->onepass)
            return bfail(nullptr, LBM_ERR_ARG, "contexts with the one-pass layout cannot join a batch");
        if (ctxs[i]->parity != ctxs[0]->parity)
            return bfail(nullptr, LBM_ERR_STATE, "all contexts must have taken an equal number of steps mod 2");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return bfail(nullptr, LBM_ERR_ARG, "a context appears twice in the batch");
    }
    lbm_batch* b = new lbm_batch();
    b->members.assign(ctxs, ctxs + n);
    b->stream = (cudaStream_t)cuda_stream;
    lbm_status s = LBM_OK;
    if (cudaMalloc((void**)&b->counter, sizeof(int)) != cudaSuccess) s = bfail(b, LBM_ERR_OOM, "batch set-up: counter");
    if (s == LBM_OK) s = regroup(b);
    if (s == LBM_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) s = bfail(b, LBM_ERR_CUDA, "batch set-up");
    if (s != LBM_OK) {
        lbm::set_thread_error(b->err.c_str());
        lbm_batch_destroy(b);
        return s;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int32_t n) {
    if (!b) return LBM_ERR_ARG;
    if (n < 0) return bfail(b, LBM_ERR_ARG, "n must be >= 0");
    const int parity = b->members[0]->parity;
    for (const lbm_ctx* c : b->members) {
        if (c->parity != parity) return bfail(b, LBM_ERR_STATE, "members were stepped apart: AA phases differ");
        if (c->sticky != LBM_OK) return bfail(b, c->sticky, "a member has a sticky error: " + c->err);
    }
    if (members_changed(b)) {   // e.g. a member was re-initialised with a solid mask: regroup
        lbm_status s = regroup(b);
        if (s != LBM_OK) return s;
    }
    int done = 0;
    if (n >= 2) {
        if (b->graph_parity != parity) {
            lbm_status s = record_graph(b, parity);
            if (s != LBM_OK) return s;
        }
        const int pairs = n / 2;
        if (b->graph_mode == 1) {
            set_counter_kernel<<<1, 1, 0, b->stream>>>(b->counter, pairs);
            BCK(b, cudaGetLastError());
            BCK(b, cudaGraphLaunch(b->exec, b->stream));
        } else {
            for (int k = 0; k < pairs; ++k) BCK(b, cudaGraphLaunch(b->exec, b->stream));
        }
        done = 2 * pairs;
    }
    if (done < n) BCK(b, step_once(b, parity, b->stream));
    advance_members(b, n);
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    BCK(b, cudaStreamSynchronize(b->stream));
    lbm_status first = LBM_OK;
    for (lbm_ctx* c : b->members) {
        lbm_status s = lbm_sync(c);
        if (s != LBM_OK && first == LBM_OK) {
            first = s;
            b->err = lbm_last_error(c);
        }
    }
    return first;
}

}  // extern "C"

namespace {

// The group with the same lattice and physics and the other solid handling (-1 if none).  A member
// with solids has its solid-free tiles in one and the others in the other; both must be cut into the
// same columns (the same tile shape), or their tiles would not partition the member's cells.
int partner_group(const lbm_batch* b, int k) {
    const Group& g = b->groups[k];
    for (int j = 0; j < (int)b->groups.size(); ++j) {
        const Group& h = b->groups[j];
        if (j != k && h.Q == g.Q && h.solids != g.solids && std::memcmp(&h.phys, &g.phys, sizeof(KParams)) == 0)
            return j;
    }
    return -1;
}

// Times every group's collide launches over `trial_steps` steps with each group set to candidate
// (shape_of(g, ci), zchunk_of(g, ci)) in turn, ci < ncand; times[ci][g] receives the total.  The
// members advance by ncand x (trial_steps + 1) steps.
template <class SF, class ZF>
lbm_status time_candidates(lbm_batch* b, int trial_steps, int ncand, SF shape_of, ZF zchunk_of,
                           std::vector<std::vector<double>>& times) {
    const size_t G = b->groups.size();
    times.assign(ncand, std::vector<double>(G, 0.0));
    std::vector<cudaEvent_t> ev(2 * G * trial_steps);
    for (auto& e : ev) BCK(b, cudaEventCreate(&e));
    lbm_status result = LBM_OK;
    for (int ci = 0; ci < ncand && result == LBM_OK; ++ci) {
        for (size_t k = 0; k < G && result == LBM_OK; ++k) {
            Group& g = b->groups[k];
            g.shape = shape_of((int)k, ci);
            g.zchunk = zchunk_of((int)k, ci);
            result = build_tiles(b, g);
        }
        if (result != LBM_OK) break;
        drop_graph(b);
        int parity = b->members[0]->parity;
        // one untimed step, then per-group events around every collide launch
        cudaError_t e = step_once(b, parity, b->stream);
        parity ^= 1;
        for (int s = 0; s < trial_steps && e == cudaSuccess; ++s) {
            for (size_t k = 0; k < G && e == cudaSuccess; ++k) {
                e = cudaEventRecord(ev[2 * (s * G + k)], b->stream);
                if (e == cudaSuccess) e = collide_group(b->groups[k], parity, b->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev[2 * (s * G + k) + 1], b->stream);
            }
            for (size_t k = 0; k < G && e == cudaSuccess; ++k) e = psi_group(b->groups[k], parity ^ 1, b->stream);
            parity ^= 1;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) {
            result = bfail(b, LBM_ERR_CUDA, std::string("tuning: ") + cudaGetErrorString(e));
            break;
        }
        advance_members(b, trial_steps + 1);
        for (size_t k = 0; k < G; ++k) {
            for (int s = 0; s < trial_steps; ++s) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[2 * (s * G + k)], ev[2 * (s * G + k) + 1]);
                times[ci][k] += ms;
            }
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return result;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_tune(lbm_batch* b, int32_t trial_steps, int32_t* zchunk_out, int32_t max_groups) {
    if (!b) return LBM_ERR_ARG;
    if (trial_steps < 1) return bfail(b, LBM_ERR_ARG, "trial_steps must be >= 1");
    const int G = (int)b->groups.size();
    std::vector<std::vector<double>> t;
    // stage 1: every tile shape (on all groups at once) with automatic z-chunks; a group and its
    // partner take the shape that minimises their summed time
    lbm_status r = time_candidates(
        b, trial_steps, lbm::BATCH_NSHAPES, [](int, int ci) { return ci; }, [](int, int) { return 0; }, t);
    if (r != LBM_OK) return r;
    std::vector<int> shape(G, 0), zchunk(G, 0);
    for (int k = 0; k < G; ++k) {
        const int p = partner_group(b, k);
        double best = 1e300;
        for (int ci = 0; ci < lbm::BATCH_NSHAPES; ++ci) {
            const double v = t[ci][k] + (p >= 0 ? t[ci][p] : 0.0);
            if (v < best) {
                best = v;
                shape[k] = ci;
            }
        }
    }
    // stage 2: the z-chunks for the chosen shapes, per group
    const int zc[] = {0, 1, 4, 8, 16, 32, ZC_WHOLE};
    const int nz = (int)(sizeof(zc) / sizeof(zc[0]));
    r = time_candidates(
        b, trial_steps, nz, [&](int k, int) { return shape[k]; }, [&](int, int ci) { return zc[ci]; }, t);
    if (r != LBM_OK) return r;
    for (int k = 0; k < G; ++k) {
        double best = 1e300;
        for (int ci = 0; ci < nz; ++ci)
            if (t[ci][k] < best) {
                best = t[ci][k];
                zchunk[k] = zc[ci];
            }
    }
    for (int k = 0; k < G; ++k) {
        b->groups[k].shape = shape[k];
        b->groups[k].zchunk = zchunk[k];
        lbm_status s = build_tiles(b, b->groups[k]);
        if (s != LBM_OK) return s;
        if (zchunk_out && k < max_groups) zchunk_out[k] = zchunk[k];
    }
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_group(const lbm_batch* b, int32_t group, int32_t* lattice, int32_t* solids, int32_t* shape,
                           int32_t* zchunk) {
    if (!b) return LBM_ERR_ARG;
    if (group < 0 || group >= (int32_t)b->groups.size()) return LBM_ERR_ARG;
    const Group& g = b->groups[group];
    if (lattice) *lattice = g.Q;
    if (solids) *solids = g.solids;
    if (shape) *shape = g.shape;
    if (zchunk) *zchunk = g.zchunk;
    return LBM_OK;
}

lbm_status lbm_batch_set_group(lbm_batch* b, int32_t group, int32_t shape, int32_t zchunk) {
    if (!b) return LBM_ERR_ARG;
    if (group < 0 || group >= (int32_t)b->groups.size()) return bfail(b, LBM_ERR_ARG, "no such group");
    if (shape < 0 || shape >= lbm::BATCH_NSHAPES) return bfail(b, LBM_ERR_ARG, "shape must lie in [0, LBM_BATCH_SHAPES)");
    if (zchunk < 0) return bfail(b, LBM_ERR_ARG, "zchunk must be >= 0");
    Group& g = b->groups[group];
    g.shape = shape;
    g.zchunk = zchunk;
    drop_graph(b);
    lbm_status s = build_tiles(b, g);
    const int p = partner_group(b, group);
    if (s == LBM_OK && p >= 0 && b->groups[p].shape != shape) {   // the partner takes the same columns
        b->groups[p].shape = shape;
        s = build_tiles(b, b->groups[p]);
    }
    return s;
}

lbm_status lbm_batch_info(const lbm_batch* b, int32_t* ngroups, int32_t* ntiles, int32_t* graph_mode) {
    if (!b) return LBM_ERR_ARG;
    if (ngroups) *ngroups = (int32_t)b->groups.size();
    if (ntiles) {
        long long t = 0;
        for (const Group& g : b->groups) t += g.ntiles;
        *ntiles = (int32_t)std::min<long long>(t, 0x7fffffff);
    }
    if (graph_mode) *graph_mode = b->graph_mode;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    (void)cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (Group& g : b->groups) free_tiles(g);
    if (b->counter) cudaFree(b->counter);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t s2 : b->side) cudaStreamDestroy(s2);
    for (cudaEvent_t ev : b->done) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : lbm_last_error(nullptr); }

}  // extern "C"
