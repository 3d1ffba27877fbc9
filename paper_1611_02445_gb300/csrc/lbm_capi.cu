// lbm_capi.cu -- the extern "C" entry points of liblbm_gb300 (declared in include/lbm.h).
//
// Host-side orchestration only: argument validation, device allocation, the order of
// kernel launches on the context's stream, and host <-> device copies. Every step of
// the computation runs in the kernels of lbm_tiles.cu and lbm_step.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_collide.cuh"
#include "lbm_internal.cuh"
#include "../../include/lbm_testing.h"

namespace lbm {
int reduce_blocks(int64_t n_tiles);
}

namespace lbm {

namespace {
std::atomic<int64_t> g_live_allocs{0};
std::atomic<int64_t> g_fail_after{-1};   // allocations left before an injected failure; < 0: none
}  // namespace

cudaError_t dmalloc(void** p, size_t bytes) {
    *p = nullptr;
    if (g_fail_after.load() >= 0 && g_fail_after.fetch_sub(1) == 0) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1);
    return e;
}

void dfree(void* p) {
    if (!p) return;
    cudaFree(p);
    g_live_allocs.fetch_sub(1);
}

}  // namespace lbm

namespace {

thread_local std::string g_create_err;

// Errors that can leave device state undefined poison the context (sticky); argument
// and ordering errors are reported and leave the context as it was.
bool is_sticky(lbm_status st) { return st == LBM_ECUDA || st == LBM_ENOMEM || st == LBM_EINTERNAL; }

lbm_status fail(lbm_ctx* c, lbm_status st, const std::string& msg) {
    if (!c) {
        g_create_err = msg;
        return st;
    }
    if (c->sticky != LBM_OK) return c->sticky;
    c->err = msg;
    if (is_sticky(st)) c->sticky = st;
    return st;
}

lbm_status cuda_fail(lbm_ctx* c, const char* what, cudaError_t e) {
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(c, call)                                         \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return cuda_fail((c), #call, _e);  \
    } while (0)

#define LBM_CHECK_CTX(c)                                          \
    do {                                                          \
        if (!(c)) return LBM_EINVAL;                              \
        if ((c)->sticky != LBM_OK) return (c)->sticky;            \
    } while (0)

bool finite3(const double* v) { return !v || (std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2])); }

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return lbm::dmalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void drop_graphs(lbm_ctx* c) {
    for (int i = 0; i < 2; i++)
        if (c->graph[i]) {
            cudaGraphExecDestroy(c->graph[i]);
            c->graph[i] = nullptr;
        }
}

// Capture GRAPH_STEPS steps starting from copy `start` on a private stream (the legacy
// default stream cannot be captured); the graph is then launched on the context stream.
cudaError_t build_graph(lbm_ctx* c, int start) {
    cudaError_t e = lbm::prepare_step(c);
    if (e != cudaSuccess) return e;
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaStream_t saved = c->stream;
    c->stream = cap;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int cur = start;
        for (int k = 0; k < lbm::GRAPH_STEPS && e == cudaSuccess; k++) {
            e = lbm::launch_step(c, c->f[cur], c->f[1 - cur]);
            cur ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    c->stream = saved;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[start], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return e;
}

void free_all(lbm_ctx* c) {
    drop_graphs(c);
    void* bufs[] = {c->tile_map, c->non_empty, c->nbr,    c->smask,  c->tflags, c->ntype,    c->nword,
                    c->groups,   c->fword,     c->fidx,   c->gfield, c->gfield_c, c->f[0], c->f[1],
                    c->partials, c->d_out, c->seed, c->tlane, c->nrec, c->frank, c->check};
    for (void* b : bufs)
        if (b) lbm::dfree(b);
    c->tile_map = nullptr;
    c->non_empty = nullptr;
    c->nbr = nullptr;
    c->smask = nullptr;
    c->tflags = nullptr;
    c->ntype = nullptr;
    c->nword = nullptr;
    c->groups = nullptr;
    c->fword = nullptr;
    c->fidx = nullptr;
    c->tlane = nullptr;
    c->nrec = nullptr;
    c->frank = nullptr;
    c->gfield_c = nullptr;
    c->f[0] = c->f[1] = nullptr;
    c->gfield = nullptr;
    c->partials = nullptr;
    c->d_out = nullptr;
    c->seed = nullptr;
    c->check = nullptr;
}

// Device-side check that every neighbour entry is -1 or a valid rank.
__global__ void k_check_nbr(const int32_t* __restrict__ nbr, int64_t n, int64_t n_tiles, int* __restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = nbr[i];
        if (v < -1 || v >= n_tiles) atomicOr(bad, 1);
    }
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct StateHeader {
    char magic[8];
    uint32_t version;
    int32_t dtype;
    int32_t nx, ny, nz;
    uint32_t periodic;
    int64_t n_tiles;
    uint64_t geometry_hash;
    uint64_t payload_bytes;
    uint64_t payload_hash;
    uint32_t rng_step;   // step counter of the stochastic rounding (LBM_F16S_SR), else 0
    uint32_t reserved;
};

lbm_status geometry_hash(lbm_ctx* c, uint64_t* out) {
    std::vector<uint8_t> nt((size_t)c->n_tiles * lbm::SLOTS);
    if (c->n_tiles > 0) {
        LBM_CUDA(c, cudaMemcpyAsync(nt.data(), c->ntype, nt.size(), cudaMemcpyDeviceToHost, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    int32_t dims[4] = {c->nx, c->ny, c->nz, (int32_t)c->periodic};
    *out = fnv1a(nt.data(), nt.size(), fnv1a(dims, sizeof(dims)));
    return LBM_OK;
}

// MRT relaxation constants of the step: rates in moment order (conserved moments 1,
// stress moments 1/tau, the others from the user's five), divided by the row norms.
void set_mrt_constants(lbm_ctx* c) {
    const double* r = c->mrt_user;   // s_e, s_eps, s_q, s_pi, s_m
    const double snu = c->tau > 0.5 ? 1.0 / c->tau : 1.0;
    const double s[lbm::Q] = {1.0, r[0], r[1], 1.0, r[2], 1.0, r[2], 1.0, r[2], snu,
                              r[3], snu, r[3], snu, snu, snu, r[4], r[4], r[4]};
    for (int k = 0; k < lbm::Q; k++) {
        const double n = (double)lbm::mrt_norm(k);
        c->p.mrt_a[k] = (1.0 - s[k]) / n;
        c->p.mrt_b[k] = (1.0 - 0.5 * s[k]) / n;
        c->p.mrt_a_f[k] = (float)c->p.mrt_a[k];
        c->p.mrt_b_f[k] = (float)c->p.mrt_b[k];
    }
}

// The checked build's error word after a run of steps: any failed index check makes the
// context fail with LBM_EINTERNAL (the kernel skipped the access it could not make). The
// normal build has no error word and returns at once.
lbm_status read_check(lbm_ctx* c) {
    if (!c->check) return LBM_OK;
    unsigned long long word = 0;
    LBM_CUDA(c, cudaMemcpyAsync(&word, c->check, sizeof(word), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (word == 0) return LBM_OK;
    static const char* what[] = {"?", "work-group header out of range", "node tile not in its group",
                                 "gather source of a pulled direction outside the population copy"};
    const unsigned code = (unsigned)(word >> 56);
    return fail(c, LBM_EINTERNAL,
                std::string("checked build: step kernel index check failed (") + what[code < 4 ? code : 0] +
                    ", code " + std::to_string(code) + ", value " + std::to_string(word & 0x00ffffffffffffffull) +
                    "); the access was skipped");
}

}  // namespace

extern "C" {

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

void lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return;
    free_all(ctx);
    delete ctx;
}

lbm_status lbm_set_stream(lbm_ctx* ctx, void* stream) {
    LBM_CHECK_CTX(ctx);
    ctx->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

// lbm_create's body. ghost_lo / ghost_hi: the box's first / last tile plane along z is a
// ghost plane of a slab context (its tiles get no work group and are not reduced).
static lbm_status create_impl(const uint8_t* node_type, int on_device, int nx, int ny, int nz, int tile,
                              lbm_dtype dtype, unsigned periodic, void* stream, int ghost_lo, int ghost_hi,
                              lbm_ctx** out) {
    g_create_err.clear();
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!node_type) return fail(nullptr, LBM_EINVAL, "node_type is NULL");
    if (tile != lbm::TILE) return fail(nullptr, LBM_EUNSUPPORTED, "only 4x4x4 tiles are supported");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "dimensions must be >= 1");
    if (dtype != LBM_F64 && dtype != LBM_F32 && dtype != LBM_F16S && dtype != LBM_F64_NATIVE &&
        dtype != LBM_F16S_SR)
        return fail(nullptr, LBM_EINVAL, "unknown dtype");
    const bool native64 = dtype == LBM_F64_NATIVE;
    if (native64) dtype = LBM_F64;
    const bool sr = dtype == LBM_F16S_SR;
    if (sr) dtype = LBM_F16S;
    if (periodic & ~7u) return fail(nullptr, LBM_EINVAL, "periodic mask has bits other than x, y, z");
    const int dims[3] = {nx, ny, nz};
    for (int a = 0; a < 3; a++)
        if ((periodic & (1u << a)) && dims[a] % lbm::TILE != 0)
            return fail(nullptr, LBM_EINVAL, "a periodic axis must be a multiple of 4");
    // widened before the rounding-up add: an axis near INT_MAX must not wrap
    const int64_t Tx = ((int64_t)nx + 3) / 4, Ty = ((int64_t)ny + 3) / 4, Tz = ((int64_t)nz + 3) / 4;
    if (Tx * Ty > 0x7fffffffll || Tx * Ty * Tz > 0x7fffffffll)   // each factor < 2^30: no overflow
        return fail(nullptr, LBM_EINVAL, "tile grid larger than 2^31 tiles");
    const int64_t nT = Tx * Ty * Tz;

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation of the context failed");
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->Tx = (int)Tx; c->Ty = (int)Ty; c->Tz = (int)Tz;
    c->periodic = periodic;
    c->dtype = dtype;
    c->native64 = native64;
    c->sr = sr;
    c->stream = static_cast<cudaStream_t>(stream);

    uint8_t* d_nt = nullptr;
    uint8_t* d_flag = nullptr;
    int64_t* d_sums = nullptr;
    int64_t* d_count = nullptr;
    int* d_bad = nullptr;
    auto cleanup = [&]() {
        if (!on_device && d_nt) lbm::dfree(d_nt);
        if (d_flag) lbm::dfree(d_flag);
        if (d_sums) lbm::dfree(d_sums);
        if (d_count) lbm::dfree(d_count);
        if (d_bad) lbm::dfree(d_bad);
    };
    auto bail = [&](lbm_status s2) {
        g_create_err = c->err.empty() ? std::string("lbm_create failed") : c->err;
        cudaStreamSynchronize(c->stream);
        cleanup();
        lbm_destroy(c);
        return s2;
    };
#define LBM_CREATE_CUDA(call)                                              \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) return bail(cuda_fail(c, #call, _e));       \
    } while (0)

    const int64_t N = (int64_t)nx * ny * nz;
    if (on_device) {
        d_nt = const_cast<uint8_t*>(node_type);
    } else {
        LBM_CREATE_CUDA(dev_alloc(&d_nt, (size_t)N));
        LBM_CREATE_CUDA(cudaMemcpyAsync(d_nt, node_type, (size_t)N, cudaMemcpyHostToDevice, c->stream));
    }
    const int64_t nb = lbm::scan_block_count(nT);
    LBM_CREATE_CUDA(dev_alloc(&c->tile_map, (size_t)nT));
    LBM_CREATE_CUDA(dev_alloc(&c->non_empty, (size_t)nT));
    LBM_CREATE_CUDA(dev_alloc(&d_flag, (size_t)nT));
    LBM_CREATE_CUDA(dev_alloc(&d_sums, (size_t)nb));
    LBM_CREATE_CUDA(dev_alloc(&d_count, 1));
    LBM_CREATE_CUDA(dev_alloc(&d_bad, 1));
    LBM_CREATE_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
    LBM_CREATE_CUDA(lbm::launch_tile_flags(d_nt, nx, ny, nz, c->Tx, c->Ty, c->Tz, d_flag, d_bad, c->stream));
    LBM_CREATE_CUDA(lbm::launch_scan_flags(d_flag, nT, c->tile_map, c->non_empty, d_count, d_sums, nb, c->stream));
    int64_t count = 0;
    int bad = 0;
    LBM_CREATE_CUDA(cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, c->stream));
    LBM_CREATE_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    LBM_CREATE_CUDA(cudaStreamSynchronize(c->stream));
    if (bad) {
        fail(c, LBM_EINVAL, "node_type holds values other than 0 (solid), 1 (fluid), 2 (inlet), 3 (outlet)");
        return bail(LBM_EINVAL);
    }
    if (count < 0 || count > nT) {
        fail(c, LBM_EINTERNAL, "tile count out of range");
        return bail(LBM_EINTERNAL);
    }
    if (count > (int64_t)(0x7fffffff / lbm::SLOTS)) {
        // per-node slot indices (tile * 64 + slot) and work-group node offsets are 32-bit
        fail(c, LBM_EUNSUPPORTED, "more than 2^31 / 64 kept tiles (2^31 node slots) are not supported");
        return bail(LBM_EUNSUPPORTED);
    }
    c->n_tiles = count;
    c->n_partials = lbm::reduce_blocks(count);
    LBM_CREATE_CUDA(dev_alloc(&c->nbr, (size_t)count * lbm::NBR_STRIDE));
    LBM_CREATE_CUDA(dev_alloc(&c->nword, (size_t)count * lbm::SLOTS));
    LBM_CREATE_CUDA(dev_alloc(&c->smask, (size_t)count));
    LBM_CREATE_CUDA(dev_alloc(&c->tflags, (size_t)count));
    LBM_CREATE_CUDA(dev_alloc(&c->ntype, (size_t)count * lbm::SLOTS));
    LBM_CREATE_CUDA(dev_alloc(&c->partials, (size_t)c->n_partials * 4));
    LBM_CREATE_CUDA(dev_alloc(&c->d_out, 8));
#ifdef LBM_CHECKED
    LBM_CREATE_CUDA(dev_alloc(&c->check, 1));
    LBM_CREATE_CUDA(cudaMemsetAsync(c->check, 0, sizeof(unsigned long long), c->stream));
#endif
    if (sr) {
        LBM_CREATE_CUDA(dev_alloc(&c->seed, 2));
        LBM_CREATE_CUDA(cudaMemsetAsync(c->seed, 0, 2 * sizeof(uint32_t), c->stream));
    }
    LBM_CREATE_CUDA(lbm::launch_tile_meta(c, d_nt));
    unsigned long long nonsolid = 0;
    LBM_CREATE_CUDA(cudaMemcpyAsync(&nonsolid, c->d_out, sizeof(nonsolid), cudaMemcpyDeviceToHost, c->stream));
    LBM_CREATE_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
    if (count > 0) {
        k_check_nbr<<<152 * 4, 256, 0, c->stream>>>(c->nbr, count * lbm::NBR_STRIDE, count, d_bad);
        LBM_CREATE_CUDA(cudaGetLastError());
    }
    LBM_CREATE_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    LBM_CREATE_CUDA(cudaStreamSynchronize(c->stream));
    if (bad) {
        fail(c, LBM_EINTERNAL, "neighbour table holds an out-of-range tile rank");
        return bail(LBM_EINTERNAL);
    }
    // only after the check above: this kernel dereferences the neighbour ranks
    LBM_CREATE_CUDA(lbm::launch_node_words(c));
    LBM_CREATE_CUDA(cudaStreamSynchronize(c->stream));
    c->n_nonsolid = (int64_t)nonsolid;
    {
        // Work units of the step kernel: consecutive tiles, at most GROUP_MAX_TILES_* of
        // them and at most GROUP_MAX_NODES (FP64: GROUP_MAX_NODES_F64) non-solid nodes, so
        // that threads map to non-solid nodes only. The host forms the groups greedily from
        // the tiles' node counts (their solid masks: 8 bytes per tile) and decides per tile
        // where its lanes and fill entries start; k_lane_lists then writes the per-lane
        // lists on the device.
        std::vector<uint64_t> smask_h((size_t)count);
        std::vector<uint32_t> tiles_h((size_t)count);
        if (count > 0) {
            LBM_CREATE_CUDA(cudaMemcpyAsync(smask_h.data(), c->smask, smask_h.size() * 8, cudaMemcpyDeviceToHost,
                                            c->stream));
            LBM_CREATE_CUDA(cudaMemcpyAsync(tiles_h.data(), c->non_empty, tiles_h.size() * 4, cudaMemcpyDeviceToHost,
                                            c->stream));
            LBM_CREATE_CUDA(cudaStreamSynchronize(c->stream));
        }
        // own tiles: kept tiles outside the ghost planes; the ranks follow the z-outermost
        // discovery order, so each plane is one contiguous range of ranks
        const int64_t plane = (int64_t)c->Tx * c->Ty;
        c->ghost_lo = ghost_lo;
        c->ghost_hi = ghost_hi;
        c->own_k0 = 0;
        c->own_k1 = count;
        c->bnd_lo = c->bnd_hi = 0;
        for (int64_t r = 0; r < count; r++) {
            const int64_t tz = (int64_t)tiles_h[r] / plane;
            if (tz < ghost_lo) c->own_k0 = r + 1;
            if (tz >= c->Tz - ghost_hi && c->own_k1 == count) c->own_k1 = r;
            if (tz == ghost_lo) c->bnd_lo++;
            if (tz == c->Tz - 1 - ghost_hi) c->bnd_hi++;
        }
        const int64_t n_own = c->own_k1 - c->own_k0;
        // Storage groups, formed greedily over the lower ghost plane, the own tiles and the
        // upper ghost plane separately (the step updates whole groups of own tiles): each
        // tile gets its padded lane tlane, and the own groups become the step's work groups.
        std::vector<int4> groups;
        std::vector<int32_t> tlane_h((size_t)count);
        std::vector<int64_t> lane0((size_t)n_own);
        std::vector<uint8_t> lt((size_t)n_own);
        const int max_nodes = dtype == LBM_F64 ? lbm::GROUP_MAX_NODES_F64 : lbm::GROUP_MAX_NODES;
        const int max_tiles = dtype == LBM_F64 ? lbm::GROUP_MAX_TILES_F64 : lbm::GROUP_MAX_TILES_4B;
        int64_t sgroups = 0, lanes = 0;
        auto form = [&](int64_t k0, int64_t k1, bool own) {
            int64_t k = k0;
            while (k < k1) {
                int4 g;
                g.x = (int)k;
                g.y = 0;
                g.z = (int)lanes;
                g.w = 0;
                while (k < k1 && g.y < max_tiles) {
                    const int cnt = lbm::SLOTS - __builtin_popcountll(smask_h[k]);
                    if (g.w + cnt > max_nodes) break;
                    tlane_h[k] = (int32_t)(sgroups * lbm::GROUP_LANES + g.w);
                    if (own) {
                        lane0[k - c->own_k0] = lanes;
                        lt[k - c->own_k0] = (uint8_t)g.y;
                        lanes += cnt;
                    }
                    g.w += cnt;
                    g.y++;
                    k++;
                }
                if (own) groups.push_back(g);
                sgroups++;
                if (sgroups > 0x7fffffffll / lbm::GROUP_LANES) return false;
            }
            return true;
        };
        bool fits = form(0, c->own_k0, false);
        c->p.sg0 = sgroups;
        fits = fits && form(c->own_k0, c->own_k1, true) && form(c->own_k1, count, false);
        if (!fits) {
            // padded lanes are 32-bit
            fail(c, LBM_EUNSUPPORTED, "more than 2^31 padded node lanes are not supported");
            return bail(LBM_EUNSUPPORTED);
        }
        // the step updates the own tiles' nodes: in a slab context fewer than the box holds
        if ((ghost_lo == 0 && ghost_hi == 0 && lanes != c->n_nonsolid) || lanes > 0x7fffffffll) {
            fail(c, LBM_EINTERNAL, "non-solid node count mismatch while building work groups");
            return bail(LBM_EINTERNAL);
        }
        c->n_own_nonsolid = lanes;
        c->n_groups = (int64_t)groups.size();
        c->n_sgroups = sgroups;
        const size_t copy_bytes = (size_t)sgroups * lbm::Q * lbm::GROUP_LANES * lbm::dtype_size(dtype);
        LBM_CREATE_CUDA(lbm::dmalloc(&c->f[0], std::max<size_t>(copy_bytes, 16)));
        LBM_CREATE_CUDA(lbm::dmalloc(&c->f[1], std::max<size_t>(copy_bytes, 16)));
        // the padding lanes of the groups are never read or written: zero, so that a saved
        // state depends on the populations alone
        LBM_CREATE_CUDA(cudaMemsetAsync(c->f[0], 0, copy_bytes, c->stream));
        LBM_CREATE_CUDA(cudaMemsetAsync(c->f[1], 0, copy_bytes, c->stream));
        LBM_CREATE_CUDA(dev_alloc(&c->tlane, (size_t)std::max<int64_t>(count, 1)));
        LBM_CREATE_CUDA(dev_alloc(&c->nrec, (size_t)std::max<int64_t>(count, 1) * lbm::NBR_STRIDE));
        LBM_CREATE_CUDA(dev_alloc(&c->groups, groups.size()));
        LBM_CREATE_CUDA(dev_alloc(&c->fword, (size_t)lanes));
        LBM_CREATE_CUDA(dev_alloc(&c->fidx, (size_t)lanes));
        LBM_CREATE_CUDA(dev_alloc(&c->frank, (size_t)lanes));
        if (count > 0) {
            LBM_CREATE_CUDA(cudaMemcpyAsync(c->tlane, tlane_h.data(), tlane_h.size() * sizeof(int32_t),
                                            cudaMemcpyHostToDevice, c->stream));
            LBM_CREATE_CUDA(lbm::launch_node_records(c));
        }
        if (!groups.empty()) {
            int64_t* d_lane0 = nullptr;
            uint8_t* d_lt = nullptr;
            cudaError_t e = dev_alloc(&d_lane0, lane0.size());
            if (e == cudaSuccess) e = dev_alloc(&d_lt, lt.size());
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->groups, groups.data(), groups.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_lane0, lane0.data(), lane0.size() * 8, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_lt, lt.data(), lt.size(), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = lbm::launch_lane_lists(c, d_lane0, d_lt);
            const cudaError_t e2 = cudaStreamSynchronize(c->stream);
            lbm::dfree(d_lane0);
            lbm::dfree(d_lt);
            LBM_CREATE_CUDA(e);
            LBM_CREATE_CUDA(e2);
        }
        LBM_CREATE_CUDA(cudaStreamSynchronize(c->stream));
    }
    c->p.omega = 1.0;
    c->p.beta = 0.5;
    c->p.rho_out = 1.0;
    c->p.n_tiles = c->n_tiles;
    c->p.n_lanes = c->n_own_nonsolid;
    c->p.n_padded = c->n_sgroups * lbm::GROUP_LANES;
    c->p.check = c->check;
    cleanup();
#undef LBM_CREATE_CUDA
    *out = c;
    return LBM_OK;
}

lbm_status lbm_create(const uint8_t* node_type, int on_device, int nx, int ny, int nz, int tile,
                      lbm_dtype dtype, unsigned periodic, void* stream, lbm_ctx** out) {
    return create_impl(node_type, on_device, nx, ny, nz, tile, dtype, periodic, stream, 0, 0, out);
}

// ------------------------------------------------------------- slabs and their halos
lbm_status lbm_partition_z(const uint8_t* node_type, int nx, int ny, int nz, int nranks, int* plane_begin) {
    g_create_err.clear();
    if (!node_type || !plane_begin) return fail(nullptr, LBM_EINVAL, "node_type and plane_begin are required");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "dimensions must be >= 1");
    const int Tz = (int)(((int64_t)nz + 3) / 4);
    if (nranks < 1 || nranks > Tz) return fail(nullptr, LBM_EINVAL, "need 1 <= nranks <= ceil(nz / 4)");
    const int64_t layer = (int64_t)nx * ny;
    std::vector<int64_t> cum((size_t)Tz + 1, 0);   // non-solid nodes below each tile plane
    for (int P = 0; P < Tz; P++) {
        int64_t cnt = 0;
        for (int64_t z = 4LL * P; z < std::min<int64_t>(4LL * P + 4, nz); z++)
            for (int64_t i = 0; i < layer; i++) cnt += node_type[z * layer + i] != 0;
        cum[P + 1] = cum[P] + cnt;
    }
    plane_begin[0] = 0;
    plane_begin[nranks] = Tz;
    for (int r = 1; r < nranks; r++) {
        // the first plane whose nodes below reach r / nranks of the total, keeping at
        // least one plane for every rank
        const double target = (double)cum[Tz] * r / nranks;
        int P = plane_begin[r - 1] + 1;
        while (P < Tz - (nranks - r) && (double)cum[P] < target) P++;
        plane_begin[r] = P;
    }
    return LBM_OK;
}

lbm_status lbm_slab_geometry(const uint8_t* node_type, int nx, int ny, int nz, unsigned periodic, int plane_begin,
                             int plane_end, uint8_t* sub, int* nz_sub, int* ghost_lo, int* ghost_hi) {
    g_create_err.clear();
    if (!node_type || !nz_sub) return fail(nullptr, LBM_EINVAL, "node_type and nz_sub are required");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "dimensions must be >= 1");
    if ((periodic & LBM_PERIODIC_Z) && nz % 4) return fail(nullptr, LBM_EINVAL, "a periodic axis must be a multiple of 4");
    const int Tz = (int)(((int64_t)nz + 3) / 4);
    if (plane_begin < 0 || plane_end > Tz || plane_begin >= plane_end)
        return fail(nullptr, LBM_EINVAL, "need 0 <= plane_begin < plane_end <= ceil(nz / 4)");
    const bool whole = plane_begin == 0 && plane_end == Tz;
    const bool pz = (periodic & LBM_PERIODIC_Z) != 0;
    const int gl = !whole && (plane_begin > 0 || pz) ? 1 : 0;
    const int gh = !whole && (plane_end < Tz || pz) ? 1 : 0;
    const int planes = plane_end - plane_begin + gl + gh;
    *nz_sub = 4 * planes;
    if (ghost_lo) *ghost_lo = gl;
    if (ghost_hi) *ghost_hi = gh;
    if (!sub) return LBM_OK;
    const int64_t layer = (int64_t)nx * ny;
    for (int q = 0; q < planes; q++) {
        const int P = ((plane_begin - gl + q) % Tz + Tz) % Tz;   // wraps only on a periodic z axis
        for (int j = 0; j < 4; j++) {
            uint8_t* dst = sub + (int64_t)(4 * q + j) * layer;
            const int64_t z = 4LL * P + j;
            if (z < nz) std::memcpy(dst, node_type + z * layer, (size_t)layer);
            else std::memset(dst, 0, (size_t)layer);                // padding: solid
        }
    }
    return LBM_OK;
}

lbm_status lbm_create_slab(const uint8_t* node_type, int nx, int ny, int nz, int tile, lbm_dtype dtype,
                           unsigned periodic, int plane_begin, int plane_end, void* stream, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    int nzs = 0, gl = 0, gh = 0;
    lbm_status st = lbm_slab_geometry(node_type, nx, ny, nz, periodic, plane_begin, plane_end, nullptr, &nzs, &gl, &gh);
    if (st != LBM_OK) return st;
    if (gl == 0 && gh == 0) return lbm_create(node_type, 0, nx, ny, nz, tile, dtype, periodic, stream, out);
    std::vector<uint8_t> sub;
    try {
        sub.resize((size_t)nx * ny * nzs);
    } catch (...) {
        return fail(nullptr, LBM_ENOMEM, "host allocation of the slab geometry failed");
    }
    lbm_slab_geometry(node_type, nx, ny, nz, periodic, plane_begin, plane_end, sub.data(), &nzs, &gl, &gh);
    // x and y keep their boundary conditions; along z the ghost planes stand for the rest
    st = create_impl(sub.data(), 0, nx, ny, nzs, tile, dtype, periodic & ~(unsigned)LBM_PERIODIC_Z, stream, gl, gh,
                     out);
    if (st == LBM_OK) (*out)->z_plane0 = plane_begin - gl;
    return st;
}

lbm_status lbm_halo_bytes(lbm_ctx* c, int side, int pack, size_t* bytes) {
    LBM_CHECK_CTX(c);
    if ((side != 0 && side != 1) || !bytes) return fail(c, LBM_EINVAL, "side must be 0 or 1, bytes non-NULL");
    const bool ghost = side == 0 ? c->ghost_lo : c->ghost_hi;
    const int64_t n = !ghost ? 0 : pack ? (side == 0 ? c->bnd_lo : c->bnd_hi)
                                        : (side == 0 ? c->own_k0 : c->n_tiles - c->own_k1);
    *bytes = (size_t)n * 5 * lbm::SLOTS * lbm::dtype_size(c->dtype);
    return LBM_OK;
}

static lbm_status halo_io(lbm_ctx* c, int side, int pack, void* buf) {
    LBM_CHECK_CTX(c);
    if (side != 0 && side != 1) return fail(c, LBM_EINVAL, "side must be 0 or 1");
    if (!(side == 0 ? c->ghost_lo : c->ghost_hi)) return fail(c, LBM_ESTATE, "no ghost plane on that side");
    if (!buf) return fail(c, LBM_EINVAL, "buf is NULL");
    if (!c->state_set) return fail(c, LBM_ESTATE, "no state");
    LBM_CUDA(c, lbm::launch_halo(c, side, pack, buf));
    return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_ctx* c, int side, void* buf) { return halo_io(c, side, 1, buf); }

lbm_status lbm_halo_unpack(lbm_ctx* c, int side, const void* buf) {
    return halo_io(c, side, 0, const_cast<void*>(buf));
}

lbm_status lbm_set_params(lbm_ctx* c, double tau, const double* g, const double* g_field,
                          int g_field_on_device, const double* u_in, double rho_out) {
    LBM_CHECK_CTX(c);
    if (!(std::isfinite(tau) && tau > 0.5)) return fail(c, LBM_EINVAL, "tau must be finite and > 1/2");
    if (!finite3(g) || !finite3(u_in)) return fail(c, LBM_EINVAL, "g and u_in must be finite");
    if (!(std::isfinite(rho_out) && rho_out > 0.0)) return fail(c, LBM_EINVAL, "rho_out must be finite and > 0");
    if (g_field) {
        const int64_t N = (int64_t)c->nx * c->ny * c->nz;
        const size_t gsize = c->dtype == LBM_F64 ? 8 : 4;
        const size_t gbytes = (size_t)std::max<int64_t>(c->n_tiles, 1) * lbm::SLOTS * gsize;
        if (!c->gfield) LBM_CUDA(c, lbm::dmalloc(&c->gfield, gbytes));
        if (!c->gfield_c) LBM_CUDA(c, lbm::dmalloc(&c->gfield_c, (size_t)std::max<int64_t>(c->n_own_nonsolid, 1) * gsize));
        const double* d_dense = g_field;
        double* tmp = nullptr;
        if (!g_field_on_device) {
            LBM_CUDA(c, dev_alloc(&tmp, (size_t)N));
            cudaError_t e = cudaMemcpyAsync(tmp, g_field, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) {
                lbm::dfree(tmp);
                return cuda_fail(c, "cudaMemcpyAsync(g_field)", e);
            }
            d_dense = tmp;
        }
        cudaError_t e = c->n_tiles > 0 ? lbm::launch_gfield(c, d_dense) : cudaSuccess;
        if (e == cudaSuccess && c->n_tiles > 0) e = lbm::launch_gfield_compact(c);
        if (tmp) {
            cudaError_t e2 = cudaStreamSynchronize(c->stream);
            lbm::dfree(tmp);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess) return cuda_fail(c, "set g_field", e);
    } else if (c->gfield) {
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
        lbm::dfree(c->gfield);
        lbm::dfree(c->gfield_c);
        c->gfield = nullptr;
        c->gfield_c = nullptr;
    }
    c->tau = tau;
    c->p.omega = 1.0 / tau;
    c->p.beta = 1.0 - 0.5 / tau;
    for (int a = 0; a < 3; a++) {
        c->p.g[a] = g ? g[a] : 0.0;
        c->p.u_in[a] = u_in ? u_in[a] : 0.0;
    }
    c->p.rho_out = rho_out;
    c->p.gfield = c->gfield;
    drop_graphs(c);   // captured launches hold the old parameters
    c->p.dfc = lbm::make_df_const(c->p.omega, c->p.beta, c->p.g[0], c->p.g[1], c->p.g[2]);
    c->p.dfb = lbm::make_df_closure(c->p.u_in, c->p.rho_out);
    c->p.omega_f = (float)c->p.omega;
    c->p.beta_f = (float)c->p.beta;
    for (int a = 0; a < 3; a++) {
        c->p.g_f[a] = (float)c->p.g[a];
        c->p.u_in_f[a] = (float)c->p.u_in[a];
    }
    c->p.rho_out_f = (float)rho_out;
    c->p.rho_out_m1_f = (float)(rho_out - 1.0);
    set_mrt_constants(c);
    c->params_set = true;
    return LBM_OK;
}

lbm_status lbm_set_bc(lbm_ctx* c, int scheme, int inlet_face, int outlet_face) {
    LBM_CHECK_CTX(c);
    if (scheme != LBM_BC_EQUILIBRIUM && scheme != LBM_BC_ZOU_HE) return fail(c, LBM_EINVAL, "unknown boundary scheme");
    if (scheme == LBM_BC_ZOU_HE) {
        for (int f : {inlet_face, outlet_face}) {
            if (f < 0 || f > 5) return fail(c, LBM_EINVAL, "faces must be 0..5");
            if (c->periodic & (1u << (f >> 1))) return fail(c, LBM_EINVAL, "a Zou-He face lies on a periodic axis");
        }
    }
    c->bc = scheme;
    c->p.bc = scheme;
    c->p.zh_face[0] = inlet_face;
    c->p.zh_face[1] = outlet_face;
    drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_set_lid(lbm_ctx* c, int face, const double* u) {
    LBM_CHECK_CTX(c);
    if (face < -1 || face > 5) return fail(c, LBM_EINVAL, "face must be -1 (none) or 0..5");
    if (face >= 0 && (c->periodic & (1u << (face >> 1)))) return fail(c, LBM_EINVAL, "the lid face's axis is periodic");
    if (face >= 0 && !finite3(u)) return fail(c, LBM_EINVAL, "u must be finite");
    const int a = face >> 1;
    const int sgn = (face & 1) ? -1 : 1;   // the link crosses the face when c_a(i) = sgn
    for (int i = 0; i < lbm::Q; i++) {
        const int ci[3] = {lbm::cx(i), lbm::cy(i), lbm::cz(i)};
        double v = 0.0;
        if (face >= 0 && ci[a] == sgn) v = 6.0 * lbm::wgt(i) * (ci[0] * u[0] + ci[1] * u[1] + ci[2] * u[2]);
        c->p.lid_c[i] = v;
        c->p.lid_c_f[i] = (float)v;
    }
    LBM_CUDA(c, lbm::launch_mark_lid(c, face));
    c->lid_face = face;
    drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_set_model(lbm_ctx* c, int equilibrium, int collision, const double* rates) {
    LBM_CHECK_CTX(c);
    if (equilibrium != LBM_EQ_QCOMPR && equilibrium != LBM_EQ_INCOMPR)
        return fail(c, LBM_EINVAL, "unknown equilibrium");
    if (collision != LBM_COLL_BGK && collision != LBM_COLL_MRT) return fail(c, LBM_EINVAL, "unknown collision");
    if (rates)
        for (int k = 0; k < 5; k++)
            if (!(std::isfinite(rates[k]) && rates[k] > 0.0 && rates[k] < 2.0))
                return fail(c, LBM_EINVAL, "MRT rates must lie in (0, 2)");
    const double defaults[5] = {1.19, 1.4, 1.2, 1.4, 1.98};
    for (int k = 0; k < 5; k++) c->mrt_user[k] = rates ? rates[k] : defaults[k];
    c->p.eq = equilibrium;
    c->p.coll = collision;
    c->gen = equilibrium != LBM_EQ_QCOMPR || collision != LBM_COLL_BGK;
    set_mrt_constants(c);
    drop_graphs(c);   // captured launches hold the old parameters and kernel
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx* c, double rho0, const double* u0) {
    LBM_CHECK_CTX(c);
    if (!(std::isfinite(rho0) && rho0 > 0.0) || !finite3(u0)) return fail(c, LBM_EINVAL, "rho0 must be > 0, u0 finite");
    const double z[3] = {0.0, 0.0, 0.0};
    if (c->n_tiles > 0) LBM_CUDA(c, lbm::launch_init(c, rho0, u0 ? u0 : z));
    if (c->seed) LBM_CUDA(c, cudaMemsetAsync(c->seed, 0, 2 * sizeof(uint32_t), c->stream));
    c->cur = 0;
    c->state_set = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int n) {
    LBM_CHECK_CTX(c);
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (!c->state_set || !c->params_set) return fail(c, LBM_ESTATE, "set parameters and a state before stepping");
    int k = 0;
    if (c->use_graphs && c->n_groups > 0 && n >= lbm::GRAPH_STEPS) {
        // launch-bound small problems: replay a captured sequence of steps
        for (; k + lbm::GRAPH_STEPS <= n; k += lbm::GRAPH_STEPS) {
            if (!c->graph[c->cur]) LBM_CUDA(c, build_graph(c, c->cur));
            LBM_CUDA(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
            // GRAPH_STEPS is even: the current copy is unchanged
        }
    }
    for (; k < n; k++) {
        LBM_CUDA(c, lbm::launch_step(c, c->f[c->cur], c->f[1 - c->cur]));
        c->cur ^= 1;
    }
    return read_check(c);
}

lbm_status lbm_step_kernel(lbm_ctx* c, int kind, int n) {
    LBM_CHECK_CTX(c);
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (kind < LBM_KERNEL_FULL || kind > LBM_KERNEL_RW) return fail(c, LBM_EINVAL, "unknown kernel kind");
    if (!c->state_set || !c->params_set) return fail(c, LBM_ESTATE, "set parameters and a state before stepping");
    for (int k = 0; k < n; k++) {
        LBM_CUDA(c, lbm::launch_step_kind(c, kind, c->f[c->cur], c->f[1 - c->cur]));
        c->cur ^= 1;
    }
    return read_check(c);
}

lbm_status lbm_reduce(lbm_ctx* c, double* mass, double* momentum) {
    LBM_CHECK_CTX(c);
    if (!c->state_set) return fail(c, LBM_ESTATE, "no state");
    double h[4] = {0.0, 0.0, 0.0, 0.0};
    if (c->n_tiles > 0) {
        LBM_CUDA(c, lbm::launch_reduce(c, c->d_out));
        LBM_CUDA(c, cudaMemcpyAsync(h, c->d_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (mass) *mass = h[0];
    if (momentum)
        for (int a = 0; a < 3; a++) momentum[a] = h[1 + a];
    if (!std::isfinite(h[0])) return fail(c, LBM_ENONFINITE, "mass is not finite");
    return LBM_OK;
}

lbm_status lbm_macroscopic(lbm_ctx* c, void* rho, void* u, int out_f64, int on_device) {
    LBM_CHECK_CTX(c);
    if (!rho || !u) return fail(c, LBM_EINVAL, "rho and u are required");
    if (!c->state_set) return fail(c, LBM_ESTATE, "no state");
    const int64_t N = (int64_t)c->nx * c->ny * c->nz;
    const size_t es = out_f64 ? 8 : 4;
    void* d_rho = rho;
    void* d_u = u;
    void* tmp = nullptr;
    if (!on_device) {
        LBM_CUDA(c, lbm::dmalloc(&tmp, (size_t)N * 4 * es));
        d_rho = tmp;
        d_u = static_cast<char*>(tmp) + (size_t)N * es;
    }
    cudaError_t e = cudaMemsetAsync(d_rho, 0, (size_t)N * es, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_u, 0, (size_t)N * 3 * es, c->stream);
    if (e == cudaSuccess) e = lbm::launch_macroscopic(c, d_rho, d_u, out_f64);
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(rho, d_rho, (size_t)N * es, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, d_u, (size_t)N * 3 * es, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (tmp) {
        if (e != cudaSuccess) cudaStreamSynchronize(c->stream);
        lbm::dfree(tmp);
    }
    if (e != cudaSuccess) return cuda_fail(c, "lbm_macroscopic", e);
    return LBM_OK;
}

lbm_status lbm_get_f_box(lbm_ctx* c, int x0, int y0, int z0, int bx, int by, int bz, double* out) {
    LBM_CHECK_CTX(c);
    if (!out || bx < 1 || by < 1 || bz < 1) return fail(c, LBM_EINVAL, "bad box");
    if (!c->state_set) return fail(c, LBM_ESTATE, "no state");
    const int64_t B = (int64_t)bx * by * bz;
    double* tmp = nullptr;
    LBM_CUDA(c, dev_alloc(&tmp, (size_t)B * lbm::Q));
    cudaError_t e = lbm::launch_get_box(c, x0, y0, z0, bx, by, bz, tmp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, (size_t)B * lbm::Q * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    lbm::dfree(tmp);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(c, "lbm_get_f_box", e);
    return LBM_OK;
}

lbm_status lbm_get_f(lbm_ctx* c, double* f_dense) {
    LBM_CHECK_CTX(c);
    return lbm_get_f_box(c, 0, 0, 0, c->nx, c->ny, c->nz, f_dense);
}

lbm_status lbm_set_f(lbm_ctx* c, const double* f_dense) {
    LBM_CHECK_CTX(c);
    if (!f_dense) return fail(c, LBM_EINVAL, "f_dense is NULL");
    const int64_t N = (int64_t)c->nx * c->ny * c->nz;
    if (c->n_tiles > 0) {
        double* tmp = nullptr;
        LBM_CUDA(c, dev_alloc(&tmp, (size_t)N * lbm::Q));
        cudaError_t e = cudaMemcpyAsync(tmp, f_dense, (size_t)N * lbm::Q * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = lbm::launch_set_dense(c, tmp);
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        lbm::dfree(tmp);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return cuda_fail(c, "lbm_set_f", e);
    }
    c->state_set = true;
    return LBM_OK;
}

lbm_status lbm_adjoint(lbm_ctx* c, int T, int ckpt_every, int plane_x, double* loss, double* dL_dg,
                       int dL_dg_on_device, double* dL_dtau) {
    LBM_CHECK_CTX(c);
    if (T < 1 || ckpt_every < 1 || !loss) return fail(c, LBM_EINVAL, "T >= 1, ckpt_every >= 1 and loss are required");
    if (plane_x < 0 || plane_x >= c->nx) return fail(c, LBM_EINVAL, "plane_x outside the box");
    if (!c->state_set || !c->params_set) return fail(c, LBM_ESTATE, "set parameters and a state first");
    if (c->sr) return fail(c, LBM_EUNSUPPORTED, "lbm_adjoint does not support stochastic rounding (LBM_F16S_SR)");
    if (c->gen) return fail(c, LBM_EUNSUPPORTED, "lbm_adjoint supports only the quasi-compressible LBGK model");
    if (c->lid_face >= 0) return fail(c, LBM_EUNSUPPORTED, "lbm_adjoint does not support a moving wall");
    if (c->bc != LBM_BC_EQUILIBRIUM) return fail(c, LBM_EUNSUPPORTED, "lbm_adjoint supports only the equilibrium closures");
    if (c->ghost_lo || c->ghost_hi) return fail(c, LBM_EUNSUPPORTED, "lbm_adjoint does not support slab contexts");
    if (c->n_tiles == 0) {
        *loss = 0.0;
        if (dL_dtau) *dL_dtau = 0.0;
        return LBM_OK;
    }
    bool started = false;
    cudaError_t e = lbm::launch_adjoint(c, T, ckpt_every, plane_x, loss, dL_dg, dL_dg_on_device, dL_dtau, &started);
    if (e == cudaErrorMemoryAllocation && !started) {
        c->err = "lbm_adjoint: not enough device memory for the checkpoints; state unchanged";
        return LBM_ENOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(c, "lbm_adjoint", e);
    return LBM_OK;
}

lbm_status lbm_get_tiles(lbm_ctx* c, int32_t* tile_map, uint32_t* non_empty, int64_t* n_tiles) {
    LBM_CHECK_CTX(c);
    if (n_tiles) *n_tiles = c->n_tiles;
    const size_t nT = (size_t)c->Tx * c->Ty * c->Tz;
    if (tile_map) LBM_CUDA(c, cudaMemcpyAsync(tile_map, c->tile_map, nT * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    if (non_empty && c->n_tiles > 0)
        LBM_CUDA(c, cudaMemcpyAsync(non_empty, c->non_empty, (size_t)c->n_tiles * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_get_info(lbm_ctx* c, int64_t* n_tiles, int64_t* n_nonsolid, int64_t* copy_bytes) {
    LBM_CHECK_CTX(c);
    if (n_tiles) *n_tiles = c->n_tiles;
    if (n_nonsolid) *n_nonsolid = c->n_own_nonsolid;
    if (copy_bytes) *copy_bytes = c->n_sgroups * lbm::Q * lbm::GROUP_LANES * (int64_t)lbm::dtype_size(c->dtype);
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* c, void* blob, size_t* nbytes) {
    LBM_CHECK_CTX(c);
    if (!nbytes) return fail(c, LBM_EINVAL, "nbytes is NULL");
    const size_t payload = (size_t)c->n_sgroups * lbm::Q * lbm::GROUP_LANES * lbm::dtype_size(c->dtype);
    const size_t total = sizeof(StateHeader) + payload;
    if (!blob) {
        *nbytes = total;
        return LBM_OK;
    }
    if (*nbytes < total) return fail(c, LBM_EINVAL, "blob too small");
    if (!c->state_set) return fail(c, LBM_ESTATE, "no state");
    StateHeader h{};
    std::memcpy(h.magic, "LBMGB300", 8);
    h.version = 3;
    h.dtype = c->dtype;
    h.nx = c->nx; h.ny = c->ny; h.nz = c->nz;
    h.periodic = c->periodic;
    h.n_tiles = c->n_tiles;
    lbm_status st = geometry_hash(c, &h.geometry_hash);
    if (st != LBM_OK) return st;
    h.payload_bytes = payload;
    char* dst = static_cast<char*>(blob) + sizeof(StateHeader);
    if (c->seed) LBM_CUDA(c, cudaMemcpyAsync(&h.rng_step, c->seed + c->cur, 4, cudaMemcpyDeviceToHost, c->stream));
    if (payload > 0) LBM_CUDA(c, cudaMemcpyAsync(dst, c->f[c->cur], payload, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    h.payload_hash = fnv1a(dst, payload);
    std::memcpy(blob, &h, sizeof(h));
    *nbytes = total;
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* c, const void* blob, size_t nbytes) {
    LBM_CHECK_CTX(c);
    if (!blob || nbytes < sizeof(StateHeader)) return fail(c, LBM_ESTATE, "blob too small");
    StateHeader h;
    std::memcpy(&h, blob, sizeof(h));
    const size_t payload = (size_t)c->n_sgroups * lbm::Q * lbm::GROUP_LANES * lbm::dtype_size(c->dtype);
    if (std::memcmp(h.magic, "LBMGB300", 8) != 0 || h.version != 3) return fail(c, LBM_ESTATE, "not a state blob");
    if (h.dtype != c->dtype || h.nx != c->nx || h.ny != c->ny || h.nz != c->nz || h.periodic != c->periodic ||
        h.n_tiles != c->n_tiles || h.payload_bytes != payload || nbytes < sizeof(h) + payload)
        return fail(c, LBM_ESTATE, "state blob is for another geometry or dtype");
    const char* src = static_cast<const char*>(blob) + sizeof(StateHeader);
    if (fnv1a(src, payload) != h.payload_hash) return fail(c, LBM_ESTATE, "state blob checksum mismatch");
    uint64_t gh = 0;
    lbm_status st = geometry_hash(c, &gh);
    if (st != LBM_OK) return st;
    if (gh != h.geometry_hash) return fail(c, LBM_ESTATE, "state blob geometry hash mismatch");
    if (payload > 0) LBM_CUDA(c, cudaMemcpyAsync(c->f[c->cur], src, payload, cudaMemcpyHostToDevice, c->stream));
    if (c->seed) LBM_CUDA(c, cudaMemcpyAsync(c->seed + c->cur, &h.rng_step, 4, cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->state_set = true;
    return LBM_OK;
}

// ---------------------------------------------------------------- test hooks
int64_t lbm_testing_live_allocations(void) { return lbm::g_live_allocs.load(); }

void lbm_testing_fail_allocation(int64_t k) { lbm::g_fail_after.store(k < 0 ? -1 : k); }

int lbm_testing_checked_build(void) {
#ifdef LBM_CHECKED
    return 1;
#else
    return 0;
#endif
}

lbm_status lbm_testing_plant_check(lbm_ctx* c, uint64_t word) {
    LBM_CHECK_CTX(c);
    if (!c->check) return fail(c, LBM_EUNSUPPORTED, "not a checked build (LBM_CHECKED)");
    const unsigned long long w = word;
    LBM_CUDA(c, cudaMemcpyAsync(c->check, &w, sizeof(w), cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

}  // extern "C"
