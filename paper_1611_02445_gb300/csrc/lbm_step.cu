// lbm_step.cu -- the fused collide-and-stream step kernel (Sec. 3.4, Algorithm 2).
//
// Work unit: a group of up to 16 (FP64) or 8 consecutive kept tiles holding up to 256 non-solid
// nodes, one thread per non-solid node (solid slots of a tile get no thread, so no warp
// lane idles on them). Persistent CTAs walk the groups b, b + G, b + 2G, ... with a
// software pipeline, so that while a group is computed the next group's gathers are
// already in flight:
//   header(g) cp.async of the group's {first tile, tiles, first node, nodes}, three
//             groups ahead, into a 4-slot ring;
//   meta(g)   cp.async of the group's neighbour records (the local tileMap copy of
//             Algorithm 2: for each of the 27 neighbour positions of a tile, the index of
//             that tile's first node), the per-node words (which directions bounce, node
//             type, tile and slot) and source ranks into shared-memory rings;
//   gather(g) every non-solid node pulls f_i from x - c_i -- its own tile's or a
//             neighbour tile's data block i -- or, when the word says the source is
//             solid, dropped or outside the box, its own A_inv(i)(x) (halfway
//             bounce-back, Sec. 2.2; propagation only between non-solid nodes,
//             Sec. 3.4): 19 cp.async copies per node into a staging slot (two for the
//             4-byte formats; one for FP64, refilled column by column as it is read), so
//             the bytes in flight do not occupy registers;
//   compute(g) the moving-wall term of lid links, inlet/outlet closures (equilibrium,
//             or Zou-He completion then collision), the collision (LBGK + Guo, Eq. 2, 3,
//             7; or the incompressible / MRT models) and coalesced stores of all 19
//             results into the other copy.
// Solid nodes have no storage and issue no copies. A work group is also a storage group:
// its nodes' values of direction i are one contiguous 256-value data block, so the
// stores of a group write whole 32-byte sectors (DRAM never reads a sector back to merge
// a partial write), and a gather reads the source node at the neighbour record of its
// tile plus the source slot's rank among that tile's non-solid slots (precomputed per
// node and direction at creation).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <type_traits>

#include "lbm_collide.cuh"
#include "lbm_internal.cuh"
#include "lbm_store.cuh"

namespace lbm {

// Threads per CTA (one per non-solid node of a work group), resident CTAs per SM and the
// tile limit of a work group, per storage format. The CTA count also sets the shared
// memory carveout, and what is left of the SM's 256 KB serves as L1 for the gathers:
//   FP16: 4 CTAs of 256 threads (44 KB of shared memory each, 60 KB of L1).
//   FP32: 3 CTAs of 256 threads (92 KB of L1; 6 % faster than 4 CTAs with 60 KB).
//   FP64: 2 CTAs of 256 threads (90 KB each, up to 128 registers); 3 CTAs of 192 threads
//         cap the registers at 96, and the double-float collision then spills (-20 %).
// Measured and not kept: 8 CTAs of 128 threads (-25 %), 2 of 512 (-1 to -2 %), groups of
// 16 tiles for the 4-byte formats (their larger neighbour staging pushes 4 CTAs past the
// 196 KB carveout, leaving 28 KB of L1: -25 %).
template <int DT> struct StepCfg {
    static constexpr int THREADS = 256;
    static constexpr int CTAS = 4;
    static constexpr int SLOTS = 2;
    static constexpr int MAX_TILES = GROUP_MAX_TILES_4B;
};
template <> struct StepCfg<LBM_F32> {
    static constexpr int THREADS = 256;
    static constexpr int CTAS = 3;
    static constexpr int SLOTS = 2;
    static constexpr int MAX_TILES = GROUP_MAX_TILES_4B;
};
template <> struct StepCfg<LBM_F64> {
    static constexpr int THREADS = 256;
    static constexpr int CTAS = 3;
    static constexpr int SLOTS = 1;
    static constexpr int MAX_TILES = GROUP_MAX_TILES_F64;
};
static_assert(StepCfg<LBM_F32>::THREADS == GROUP_MAX_NODES && StepCfg<LBM_F64>::THREADS == GROUP_MAX_NODES_F64,
              "work groups and CTAs must agree");
constexpr int HDR_SLOTS = 4;
constexpr int META_SLOTS = 3;
constexpr int REC_SLOTS = 2;

// ---------------------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8_sa(unsigned sa, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4_sa(unsigned sa, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ------------------------------------------------------------------- checked build
// With LBM_CHECKED every index the step takes from its tables is tested before use; a
// failed test records (code << 56) | value in the context's error word (the first one
// wins) and the access is skipped, so no out-of-range address is formed. Without it
// check_ok is constant true and the tests compile away.
__device__ __forceinline__ bool check_ok(bool ok, unsigned code, int64_t value, const StepParams& p) {
#ifdef LBM_CHECKED
    if (!ok && p.check)
        atomicCAS(p.check, 0ull, ((unsigned long long)code << 56) | ((unsigned long long)value & 0x00ffffffffffffffull));
    return ok;
#else
    (void)ok;
    (void)code;
    (void)value;
    (void)p;
    return true;
#endif
}

// A work group's header as the stages use it: in the checked build a header outside
// the context's arrays is recorded and replaced by an empty group.
template <int DT>
__device__ __forceinline__ int4 group_header(const int4 h, const StepParams& p) {
    const bool ok = h.x >= 0 && h.y >= 0 && h.y <= StepCfg<DT>::MAX_TILES && (int64_t)h.x + h.y <= p.n_tiles &&
                    h.z >= 0 && h.w >= 0 && h.w <= StepCfg<DT>::THREADS && (int64_t)h.z + h.w <= p.n_lanes;
    return check_ok(ok, CHECK_HEADER, h.x, p) ? h : make_int4(0, 0, 0, 0);
}

// Staged element: the stored element for F64/F32; for F16S the aligned 32-bit word that
// holds the wanted half (cp.async moves at least 4 bytes), with the half picked later.
template <int DT> struct Staged { using E = uint32_t; };
template <> struct Staged<LBM_F64> { using E = uint64_t; };

template <int DT>
struct StepSmem {
    using E = typename Staged<DT>::E;
    using G = typename Store<DT>::R;
    int4 hdr[HDR_SLOTS];                                   // {t0, tiles, f0, nodes}
    // neighbour records (index of each neighbour's first node) and the nodes' source ranks:
    // read only when the group's gathers are issued, one iteration after they land
    int64_t rec[REC_SLOTS][StepCfg<DT>::MAX_TILES][NBR_STRIDE];
    uint4 rank[REC_SLOTS][StepCfg<DT>::THREADS];
    uint32_t word[META_SLOTS][StepCfg<DT>::THREADS];
    // F16S: bit i set when direction i's value is the upper half of its staged word
    uint32_t odd[StepCfg<DT>::SLOTS][DT == LBM_F16S ? StepCfg<DT>::THREADS : 1];
    // staging slots: column t of a slot holds thread t's 19 gathered values, written and
    // read by that thread alone. With one slot the next group's gathers go into the column
    // as soon as the thread has read the current values into registers; with two they go
    // into the other slot.
    E data[StepCfg<DT>::SLOTS][Q][StepCfg<DT>::THREADS];
    // last, so that a launch without a per-node force field leaves it out of the dynamic
    // shared memory (the space goes to the L1 cache, which serves the 4-byte gathers)
    G gf[META_SLOTS][StepCfg<DT>::THREADS];
};

__device__ __forceinline__ void issue_hdr(int4* hdr, int64_t grp, int64_t n_groups, const int4* __restrict__ groups) {
    if (threadIdx.x == 0 && grp < n_groups) cp_async16(hdr, groups + grp);
}

// Neighbour records of the group's tiles and the words (and forces) of its nodes.
template <int DT>
__device__ __forceinline__ void issue_meta(StepSmem<DT>& sm, int mslot, int rslot, const int4 h,
                                           const int64_t* __restrict__ nrec, const uint32_t* __restrict__ fword,
                                           const uint4* __restrict__ frank, const void* gfield_c) {
    const int t = threadIdx.x;
    constexpr int CH = NBR_STRIDE / 2;   // 16-byte chunks of a tile's records
    for (int j = t; j < h.y * CH; j += StepCfg<DT>::THREADS)
        cp_async16(&sm.rec[rslot][j / CH][2 * (j % CH)], nrec + ((int64_t)h.x + j / CH) * NBR_STRIDE + 2 * (j % CH));
    if (t < h.w) {
        cp_async4(&sm.word[mslot][t], fword + h.z + t);
        cp_async16(&sm.rank[rslot][t], frank + h.z + t);
        if (gfield_c) {
            const typename Store<DT>::R* g = static_cast<const typename Store<DT>::R*>(gfield_c);
            if (DT == LBM_F64) cp_async8(&sm.gf[mslot][t], g + h.z + t);
            else cp_async4(&sm.gf[mslot][t], g + h.z + t);
        }
    } else {
        sm.word[mslot][t] = 0;   // no node: idle thread
    }
}

// Issue the 19 gathers of this thread's node (for F16S the aligned 32-bit word that holds
// the wanted half). sg: the group's storage group; the node's own padded lane is
// 256 sg + t. dep is zero, computed from the values the thread has just read out of its
// staging column, and added to the column's shared address, so that no copy into the
// column is issued before those reads are done. A pull of direction i reads entry
// 13 + dx + 3 dy + 9 dz of the tile's neighbour records, dx = -1 for c_x = +1 at x = 0 and
// +1 for c_x = -1 at x = 3 (likewise y, z): the six byte offsets of those entries are
// formed once per node.
// I32: every element index of a copy is below 2^31 (n_padded * 19 < 2^31, up to 113 M
// non-solid nodes), so the indices are formed in 32 bits, the neighbour records read as
// their low words, and each address is one widening multiply-add (2 % faster than the
// 64-bit arithmetic, which larger contexts take).
template <int DT, int MODE, bool I32>
__device__ __forceinline__ void issue_gather(StepSmem<DT>& sm, int mslot, int rslot, int dslot, const int4 h, int64_t sg,
                                             const typename Store<DT>::T* __restrict__ A, const StepParams& p,
                                             uint32_t dep) {
    const int t = threadIdx.x;
    const uint32_t w = sm.word[mslot][t];
    if (((w >> WORD_TYPE_SHIFT) & 3u) == LBM_SOLID) return;
    const int lt = (int)((w >> WORD_LT_SHIFT) & (uint32_t)WORD_LT_MASK), s = (int)((w >> WORD_SLOT_SHIFT) & 63u);
    if (!check_ok(lt < h.y, CHECK_OWN_TILE, (int64_t)h.z + t, p)) return;
    const int x = s & 3, y = (s >> 2) & 3, z = s >> 4;
    using IX = typename std::conditional<I32, int32_t, int64_t>::type;
    const IX own = (IX)(sg * (Q * GROUP_LANES)) + t;
    const uint4 rk = sm.rank[rslot][t];
    uint32_t odd = 0;
    // byte offsets, from the record of the own tile (entry 13), of the neighbour records a
    // pull along each axis reaches: c = +1 reads the tile at a - 1, c = -1 the one at a + 1
    const char* r13 = reinterpret_cast<const char*>(&sm.rec[rslot][lt][13]);
    const int oxm = ((x - 1) >> 2) * 8, oxp = ((x + 1) >> 2) * 8;
    const int oym = ((y - 1) >> 2) * 24, oyp = ((y + 1) >> 2) * 24;
    const int ozm = ((z - 1) >> 2) * 72, ozp = ((z + 1) >> 2) * 72;
    // shared address of this thread's staging column; dep orders the copies after the reads
    const unsigned sdst = (unsigned)__cvta_generic_to_shared(&sm.data[dslot][0][t]) + dep;
    constexpr unsigned ROW = StepCfg<DT>::THREADS * sizeof(typename Staged<DT>::E);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        IX rel;   // source index minus 256 i
        if (MODE == STEP_RW || i == 0) {
            rel = own;
        } else {
            const int off = (cx(i) > 0 ? oxm : cx(i) < 0 ? oxp : 0) + (cy(i) > 0 ? oym : cy(i) < 0 ? oyp : 0) +
                            (cz(i) > 0 ? ozm : cz(i) < 0 ? ozp : 0);
            const IX nrel = *reinterpret_cast<const IX*>(r13 + off) + (IX)rank_of(rk, i);   // I32: the low word
            rel = ((w >> i) & 1) ? own + (inv(i) - i) * GROUP_LANES : nrel;
            if (!check_ok(rel + i * GROUP_LANES >= 0 && rel + i * GROUP_LANES < p.n_padded * Q, CHECK_NEIGHBOUR,
                          ((int64_t)(h.x + lt) << 8) | ((13 + off / 8) << 2), p))
                continue;
        }
        const IX src = rel + i * GROUP_LANES;
        if (DT == LBM_F64) {
            cp_async8_sa(sdst + i * ROW, A + src);
        } else if (DT == LBM_F32) {
            cp_async4_sa(sdst + i * ROW, A + src);
        } else {
            odd |= (uint32_t)(src & 1) << i;
            cp_async4_sa(sdst + i * ROW, A + (src & ~(IX)1));
        }
    }
    if (DT == LBM_F16S) sm.odd[dslot][DT == LBM_F16S ? t : 0] = odd;
}

// FP16 store of a node's 19 results h (FP32, unscaled) that keeps the node's mass and
// momentum. Rounding each value to the nearest binary16 leaves residues
// r_i = h_i - stored_i. Their sums over the node (mass sum r_i, momentum sum c_i r_i) are
// what the collision cannot relax: they persist from step to step like a small spurious
// source and force, while residues in the other moments decay. So the twelve diagonal
// directions are rounded first. Each axis' momentum residue r is then carried into that
// axis' two directions, +r/2 into the one along the axis and -r/2 into the opposite
// one, which adds r to the momentum and nothing to the mass or the momentum flux. The
// rest population 0, last, takes the mass residue. The stored node's momentum then
// differs from the computed one by at most one binary16 spacing of its axis
// populations per axis, and its mass by half a spacing of h_0.
__device__ __forceinline__ void store_f16_conserving(const float v[Q], __half* __restrict__ dst) {
    float rx = 0.f, ry = 0.f, rz = 0.f, m = 0.f;
    auto put = [&](int i, float target) {
        const __half q = __float2half_rn(target * F16_SCALE);
        dst[i * GROUP_LANES] = q;
        const float r = v[i] - __half2float(q) * F16_INV_SCALE;
        m += r;
        if (cx(i)) rx += cx(i) > 0 ? r : -r;
        if (cy(i)) ry += cy(i) > 0 ? r : -r;
        if (cz(i)) rz += cz(i) > 0 ? r : -r;
    };
#pragma unroll
    for (int i = 7; i < Q; i++) put(i, v[i]);
    const float hx = 0.5f * rx, hy = 0.5f * ry, hz = 0.5f * rz;
    put(1, v[1] + hx);
    put(3, v[3] - hx);
    put(2, v[2] + hy);
    put(4, v[4] - hy);
    put(5, v[5] + hz);
    put(6, v[6] - hz);
    put(0, v[0] + m);
}

// Read this thread's staged values of group g into registers, let `next` issue the
// gathers of the thread's node in the next group into the same column, then collide
// and store. A thread without a node in g still calls next.
template <int DT, bool VAR, int MODE, bool GEN, bool XF, typename Next>
__device__ __forceinline__ void compute_store(StepSmem<DT>& sm, int mslot, int dslot, const int4 h, int64_t sg,
                                              typename Store<DT>::T* __restrict__ B, const StepParams& p,
                                              bool has_gf, uint32_t key, Next&& next) {
    using R = typename Store<DT>::R;
    using T = typename Store<DT>::T;
    const int t = threadIdx.x;
    const uint32_t w = sm.word[mslot][t];
    const int type = (int)((w >> WORD_TYPE_SHIFT) & 3u);
    if (type == LBM_SOLID) {
        next(0u);
        return;
    }
    const int lt = (int)((w >> WORD_LT_SHIFT) & (uint32_t)WORD_LT_MASK), s = (int)((w >> WORD_SLOT_SHIFT) & 63u);
    R v[Q];
    const uint32_t odd = DT == LBM_F16S ? sm.odd[dslot][DT == LBM_F16S ? t : 0] : 0u;
    uint32_t fold = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if constexpr (DT == LBM_F16S) {
            const uint32_t word = (uint32_t)sm.data[dslot][i][t];
            fold ^= word;
            // both halves converted, the wanted one selected (2 % faster than shifting the
            // word by the half's offset first); the value is to_arith's
            const __half2 h2 = *reinterpret_cast<const __half2*>(&word);
            const float lo = __low2float(h2), hi = __high2float(h2);
            v[i] = ((odd >> i) & 1u ? hi : lo) * F16_INV_SCALE;
        } else {
            const typename Staged<DT>::E raw = sm.data[dslot][i][t];
            fold ^= (uint32_t)raw;
            v[i] = to_arith<DT>(*reinterpret_cast<const T*>(&raw), i);
        }
    }
    // one slot: 0 (p.zero is 0, unknown to the compiler), but only once every value above
    // has arrived in its register
    next(StepCfg<DT>::SLOTS == 1 ? fold & p.zero : 0u);
    const R Fx = has_gf ? sm.gf[mslot][t] : par<R>(p.g[0], p.g_f[0]);
    const R Fy = par<R>(p.g[1], p.g_f[1]), Fz = par<R>(p.g[2], p.g_f[2]);
    if (MODE == STEP_FULL && ((w >> WORD_LID_BIT) & 1u)) {
        // moving wall: bounced links that cross the lid face gain 6 w_i (c_i . u_lid)
#pragma unroll
        for (int i = 1; i < Q; i++)
            if ((w >> i) & 1u) v[i] += par<R>(p.lid_c[i], p.lid_c_f[i]);
    }
    if constexpr (MODE != STEP_FULL) {
        // calibration kernels: no collision, the gathered values are stored as they are
    } else if constexpr (GEN) {
        // incompressible equilibrium or MRT; for FP64 storage the incompressible LBGK of a
        // fluid node takes the hybrid collision as well
        if constexpr (DT == LBM_F64 && !VAR) {
            if (type == LBM_FLUID && p.coll == LBM_COLL_BGK && p.eq == LBM_EQ_INCOMPR)
                collide_df<false, true>(v, (double)Fx, p.dfc, !has_gf);
            else
                collide_model<R, false>(v, type, p, Fx, Fy, Fz);
        } else {
            collide_model<R, Store<DT>::SHIFT>(v, type, p, Fx, Fy, Fz);
        }
    } else if constexpr (DT == LBM_F64 && !VAR) {
        // FP64 storage: double-float collision for fluid nodes (and Zou-He boundary nodes
        // once completed), and the equilibrium closures of inlet and outlet nodes in the
        // same hybrid arithmetic
        int ct = type;
        if (ct != LBM_FLUID && p.bc == LBM_BC_ZOU_HE) {
            zou_he<double, false>(v, ct, p);
            ct = LBM_FLUID;
        }
        if (ct == LBM_FLUID) collide_df<XF>(v, (double)Fx, p.dfc, !has_gf);
        else closure_df(v, ct, (double)Fx, p.dfc, p.dfb, !has_gf);
    } else {
        collide<R, Store<DT>::SHIFT>(v, type, p, Fx, Fy, Fz);
    }
    if (!check_ok(lt < h.y, CHECK_OWN_TILE, (int64_t)h.z + t, p)) return;
    const int64_t own = sg * (Q * GROUP_LANES) + t;
    if constexpr (DT == LBM_F16S && VAR && MODE == STEP_FULL) {
        // stochastic rounding: two 16-bit dithers per hash of (key, node, pair)
        const uint32_t node = fmix32(key ^ (uint32_t)((h.x + lt) * SLOTS + s));
#pragma unroll
        for (int i = 0; i < Q; i += 2) {
            const uint32_t r = fmix32(node + (uint32_t)(i >> 1) * 0x9e3779b9u);
            B[own + i * GROUP_LANES] = half_dithered(v[i] * F16_SCALE, r & 0xffffu);
            if (i + 1 < Q) B[own + (i + 1) * GROUP_LANES] = half_dithered(v[i + 1] * F16_SCALE, r >> 16);
        }
    } else if constexpr (DT == LBM_F16S && MODE == STEP_FULL) {
        store_f16_conserving(v, B + own);
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) B[own + i * GROUP_LANES] = to_store<DT>(v[i], i);
    }
}

static_assert(LBM_INLET == 2 && LBM_OUTLET == 3, "closure_df takes the node types by value");

// Resident CTAs per SM of a step instantiation: the collision models (GEN) of the FP64
// format need more registers than 3 CTAs leave, and run 2.
template <int DT, bool GEN>
constexpr int step_ctas() {
    return DT == LBM_F64 && GEN ? 2 : StepCfg<DT>::CTAS;
}

// XF: the FP64 hybrid collision's form for a force along x (F_y = F_z = 0; collide_df).
// I32: 32-bit gather indices (issue_gather).
template <int DT, bool VAR, int MODE, bool GEN, bool XF, bool I32>
__global__ void __launch_bounds__(StepCfg<DT>::THREADS, step_ctas<DT, GEN>())
k_step(const typename Store<DT>::T* __restrict__ A, typename Store<DT>::T* __restrict__ B,
       const int4* __restrict__ groups, const int64_t* __restrict__ nrec, const uint32_t* __restrict__ fword,
       const uint4* __restrict__ frank, const void* __restrict__ gfield_c, int64_t n_groups, StepParams p, const uint32_t* __restrict__ seed_in,
       uint32_t* __restrict__ seed_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepSmem<DT>& sm = *reinterpret_cast<StepSmem<DT>*>(smem_raw);
    const int64_t G = gridDim.x;
    const int64_t g0 = blockIdx.x;
    uint32_t key = 0;
    if (DT == LBM_F16S && VAR) {
        // step counter of the rounding hash: read from this launch's copy, advanced into
        // the other copy's, which no thread of this launch reads
        const uint32_t t = *seed_in;
        if (blockIdx.x == 0 && threadIdx.x == 0) *seed_out = t + 1u;
        key = fmix32(t * 0x9e3779b9u + 0x7f4a7c15u);
    }
    if (g0 >= n_groups) return;
    const bool has_gf = gfield_c != nullptr;
    // prologue: headers of groups 0..2, meta of groups 0..1, gathers of group 0
    issue_hdr(&sm.hdr[0], g0, n_groups, groups);
    cp_async_commit();
    issue_hdr(&sm.hdr[1], g0 + G, n_groups, groups);
    cp_async_commit();
    issue_hdr(&sm.hdr[2], g0 + 2 * G, n_groups, groups);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    issue_meta<DT>(sm, 0, 0, group_header<DT>(sm.hdr[0], p), nrec, fword, frank, gfield_c);
    cp_async_commit();
    if (g0 + G < n_groups) issue_meta<DT>(sm, 1, 1, group_header<DT>(sm.hdr[1], p), nrec, fword, frank, gfield_c);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    issue_gather<DT, MODE, I32>(sm, 0, 0, 0, group_header<DT>(sm.hdr[0], p), p.sg0 + g0, A, p, 0u);
    cp_async_commit();
    constexpr int NS = StepCfg<DT>::SLOTS;
    int it = 0;
    for (int64_t g = g0; g < n_groups; g += G, it++) {
        if constexpr (NS == 2) {
            // pending: header(g + 2G) [done], meta(g + G), gather(g)
            cp_async_wait<1>();
            __syncthreads();   // header(g + 2G), meta(g + G) visible; iteration it - 1 finished
        } else {
            cp_async_wait<0>();
            __syncthreads();   // header(g + 2G), meta(g + G), gather(g) landed; iteration it - 1 finished
        }
        issue_hdr(&sm.hdr[(it + 3) & 3], g + 3 * G, n_groups, groups);
        cp_async_commit();
        if (g + 2 * G < n_groups)
            issue_meta<DT>(sm, (it + 2) % META_SLOTS, it & 1, group_header<DT>(sm.hdr[(it + 2) & 3], p), nrec, fword,
                           frank, gfield_c);
        cp_async_commit();
        auto gather_next = [&](uint32_t dep) {
            if (g + G < n_groups)
                issue_gather<DT, MODE, I32>(sm, (it + 1) % META_SLOTS, (it + 1) & 1, (it + 1) % NS,
                                       group_header<DT>(sm.hdr[(it + 1) & 3], p), p.sg0 + g + G, A, p, dep);
            cp_async_commit();
        };
        const int4 h = group_header<DT>(sm.hdr[it & 3], p);
        if constexpr (NS == 2) {
            // the next group's gathers go into the other slot before this group's are awaited
            gather_next(0u);
            cp_async_wait<3>();   // pending: gather(g), header(g + 3G), meta(g + 2G), gather(g + G)
            compute_store<DT, VAR, MODE, GEN, XF>(sm, it % META_SLOTS, it % NS, h, p.sg0 + g, B, p, has_gf, key,
                                              [](uint32_t) {});
        } else {
            // one slot: each thread refills its column once it has read it
            compute_store<DT, VAR, MODE, GEN, XF>(sm, it % META_SLOTS, 0, h, p.sg0 + g, B, p, has_gf, key, gather_next);
        }
    }
    cp_async_wait<0>();
}

// Shared memory of a launch: the whole StepSmem with a per-node force field, without its
// force staging (the last member) otherwise.
template <int DT>
static size_t step_smem(bool with_gf) {
    return with_gf ? sizeof(StepSmem<DT>) : offsetof(StepSmem<DT>, gf);
}

// Persistent grid of step_ctas CTAs per SM. Shared memory and L1 share one array per
// SM; the kernel's preferred carveout is set to what those CTAs need (with the force
// staging, the larger case) so that the rest stays L1, which serves the 4-byte gathers
// (cp.async.ca). Left to itself the driver picks the carveout for the highest occupancy:
// a light kernel (the calibration kinds) would fit a fifth CTA and keep 28 KB of L1
// instead of 60 KB, and run 25 % slower.
template <int DT, bool VAR, int MODE, bool GEN, bool XF, bool I32>
static int step_grid(int64_t n_groups, bool with_gf) {
    static int per_sm[2] = {-1, -1}, n_sm = 0;
    int& ps = per_sm[with_gf ? 1 : 0];
    if (ps < 0) {
        int dev = 0, smem_sm = 0, reserved = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        cudaFuncSetAttribute(k_step<DT, VAR, MODE, GEN, XF, I32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(StepSmem<DT>));
        if (smem_sm > 0) {
            const double need = (double)step_ctas<DT, GEN>() * (double)(sizeof(StepSmem<DT>) + (size_t)reserved);
            const int pct = std::min(100, std::max(1, (int)std::ceil(100.0 * need / smem_sm)));
            cudaFuncSetAttribute(k_step<DT, VAR, MODE, GEN, XF, I32>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        }
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_step<DT, VAR, MODE, GEN, XF, I32>, StepCfg<DT>::THREADS,
                                                      step_smem<DT>(with_gf));
        ps = std::max(1, std::min(ps, step_ctas<DT, GEN>()));
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(n_groups, (int64_t)ps * n_sm));
}

// 32-bit gather indices when every element index of a copy fits (issue_gather).
static bool idx32(const lbm_ctx* c) { return c->p.n_padded * (int64_t)Q < (int64_t(1) << 31); }

template <int DT, bool VAR, int MODE, bool GEN, bool XF, bool I32>
static cudaError_t launch_step_ix(lbm_ctx* c, const void* A, void* B) {
    using T = typename Store<DT>::T;
    const bool with_gf = c->gfield != nullptr;
    const int grid = step_grid<DT, VAR, MODE, GEN, XF, I32>(c->n_groups, with_gf);
    // the copy read decides which counter is read and which is advanced
    const int from = A == c->f[0] ? 0 : 1;
    const uint32_t* seed_in = c->seed ? c->seed + from : nullptr;
    uint32_t* seed_out = c->seed ? c->seed + (1 - from) : nullptr;
    k_step<DT, VAR, MODE, GEN, XF, I32><<<grid, StepCfg<DT>::THREADS, step_smem<DT>(with_gf), c->stream>>>(
        (const T*)A, (T*)B, c->groups, c->nrec, c->fword, c->frank, c->gfield ? c->gfield_c : nullptr, c->n_groups, c->p,
        seed_in, seed_out);
    return cudaGetLastError();
}

template <int DT, bool VAR, int MODE, bool GEN, bool XF>
static cudaError_t launch_step_xf(lbm_ctx* c, const void* A, void* B) {
    return idx32(c) ? launch_step_ix<DT, VAR, MODE, GEN, XF, true>(c, A, B)
                    : launch_step_ix<DT, VAR, MODE, GEN, XF, false>(c, A, B);
}

// The instantiations with the hybrid FP64 collision (FP64 storage, hybrid arithmetic,
// LBGK, fused step) have a form for a force along x, taken when F_y = F_z = 0.
template <int DT, bool VAR, int MODE, bool GEN>
constexpr bool has_xf_form() {
    return DT == LBM_F64 && !VAR && MODE == STEP_FULL && !GEN;
}
static bool force_along_x(const lbm_ctx* c) { return c->p.g[1] == 0.0 && c->p.g[2] == 0.0; }

template <int DT, bool VAR, int MODE, bool GEN>
static cudaError_t launch_step_dt(lbm_ctx* c, const void* A, void* B) {
    if constexpr (has_xf_form<DT, VAR, MODE, GEN>()) {
        if (force_along_x(c)) return launch_step_xf<DT, VAR, MODE, GEN, true>(c, A, B);
    }
    return launch_step_xf<DT, VAR, MODE, GEN, false>(c, A, B);
}

template <int DT, bool VAR, bool GEN, bool I32>
static void prepare_ix(lbm_ctx* c) {
    if constexpr (has_xf_form<DT, VAR, STEP_FULL, GEN>())
        step_grid<DT, VAR, STEP_FULL, GEN, true, I32>(1, c->gfield != nullptr);
    step_grid<DT, VAR, STEP_FULL, GEN, false, I32>(1, c->gfield != nullptr);
}

template <int DT, bool VAR, bool GEN>
static void prepare_dt(lbm_ctx* c) {
    if (idx32(c)) prepare_ix<DT, VAR, GEN, true>(c);
    else prepare_ix<DT, VAR, GEN, false>(c);
}

template <int MODE, bool GEN>
static cudaError_t launch_step_model(lbm_ctx* c, const void* A, void* B) {
    switch (c->dtype) {
        case LBM_F64:
            return c->native64 ? launch_step_dt<LBM_F64, true, MODE, GEN>(c, A, B)
                               : launch_step_dt<LBM_F64, false, MODE, GEN>(c, A, B);
        case LBM_F32: return launch_step_dt<LBM_F32, false, MODE, GEN>(c, A, B);
        default:
            return c->sr ? launch_step_dt<LBM_F16S, true, MODE, GEN>(c, A, B)
                         : launch_step_dt<LBM_F16S, false, MODE, GEN>(c, A, B);
    }
}

// The calibration kernels have no collision, so only the fused step has model variants.
template <int MODE>
static cudaError_t launch_step_mode(lbm_ctx* c, const void* A, void* B) {
    if (MODE == STEP_FULL && c->gen) return launch_step_model<STEP_FULL, true>(c, A, B);
    return launch_step_model<MODE, false>(c, A, B);
}

cudaError_t launch_step(lbm_ctx* c, const void* A, void* B) { return launch_step_kind(c, STEP_FULL, A, B); }

// One-time kernel attributes and occupancy query of the fused step, done outside any
// stream capture.
template <bool GEN>
static void prepare_model(lbm_ctx* c) {
    switch (c->dtype) {
        case LBM_F64:
            if (c->native64) prepare_dt<LBM_F64, true, GEN>(c);
            else prepare_dt<LBM_F64, false, GEN>(c);
            break;
        case LBM_F32: prepare_dt<LBM_F32, false, GEN>(c); break;
        default:
            if (c->sr) prepare_dt<LBM_F16S, true, GEN>(c);
            else prepare_dt<LBM_F16S, false, GEN>(c);
    }
}

cudaError_t prepare_step(lbm_ctx* c) {
    if (c->gen) prepare_model<true>(c);
    else prepare_model<false>(c);
    return cudaGetLastError();
}

cudaError_t launch_step_kind(lbm_ctx* c, int kind, const void* A, void* B) {
    if (c->n_groups == 0) return cudaSuccess;
    switch (kind) {
        case STEP_PROPAGATE: return launch_step_mode<STEP_PROPAGATE>(c, A, B);
        case STEP_RW: return launch_step_mode<STEP_RW>(c, A, B);
        default: return launch_step_mode<STEP_FULL>(c, A, B);
    }
}

}  // namespace lbm
