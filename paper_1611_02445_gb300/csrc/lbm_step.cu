// lbm_step.cu -- the fused collide-and-stream step kernel (Sec. 3.4, Algorithm 2).
//
// Work unit: a group of up to 8 consecutive kept tiles holding up to 256 non-solid
// nodes, one thread per non-solid node (solid slots of a tile get no thread, so no warp
// lane idles on them). Persistent CTAs walk the groups b, b + G, b + 2G, ... with a
// software pipeline, so that while a group is computed the next group's gathers are
// already in flight:
//   header(g) cp.async of the group's {first tile, tiles, first node, nodes}, three
//             groups ahead, into a 4-slot ring;
//   meta(g)   cp.async of the group's neighbour records (the local tileMap copy of
//             Algorithm 2, 28 ranks per tile) and per-node words (which directions
//             bounce, node type, tile and slot) into a 3-slot shared-memory ring;
//   gather(g) every non-solid node pulls f_i from x - c_i -- its own tile's or a
//             neighbour tile's data block i -- or, when the word says the source is
//             solid, dropped or outside the box, its own A_inv(i)(x) (halfway
//             bounce-back, Sec. 2.2; propagation only between non-solid nodes,
//             Sec. 3.4): 19 cp.async copies per node into a 2-slot staging ring, so
//             the bytes in flight do not occupy registers;
//   compute(g) moments, inlet/outlet closures or LBGK + Guo collision (Eq. 2, 3, 7)
//             and coalesced stores of all 19 results into the other copy.
// Solid nodes issue no copies and no stores.
#include <algorithm>

#include "lbm_internal.cuh"
#include "lbm_store.cuh"

namespace lbm {

constexpr int STEP_THREADS = GROUP_MAX_NODES;   // 256: one thread per non-solid node
constexpr int HDR_SLOTS = 4;
constexpr int META_SLOTS = 3;
constexpr int DATA_SLOTS = 2;

// LBGK + Guo update of one direction pair (i, inv(i)) with lattice velocity c = c_i.
// Works on f (SHIFT = false, D = rho) or on h = f - w (SHIFT = true, D = rho - 1):
//   f^eq_i - w_i (if shifted) = w (D + rho (3 cu + 4.5 cu^2 - 1.5 u.u))      (Eq. 3)
//   S_i = beta w (3 (c - u).F + 9 (c.u)(c.F))                               (Guo)
//   v*_i = (1 - omega) v_i + omega v^eq_i + S_i                              (Eq. 7)
// split into the parts even (E, Se) and odd (O, So) in c.
template <typename R>
__device__ __forceinline__ void bgk_pair(R& a, R& b, R w, R cu, R cF, R D, R rho, R uu15, R uF3,
                                         R omega, R om1, R beta) {
    const R E = w * D + (w * rho) * (R(4.5) * cu * cu - uu15);
    const R O = R(3) * (w * rho) * cu;
    const R bw = beta * w;
    const R Se = bw * (R(9) * cu * cF - uF3);
    const R So = R(3) * bw * cF;
    a = om1 * a + (omega * (E + O) + (Se + So));
    b = om1 * b + (omega * (E - O) + (Se - So));
}

// The same update on h = f - w written with j' = rho u = j + F/2 (SHIFT = true):
//   h^eq_i = w (D + 3 c.j' + (4.5 (c.j')^2 - 1.5 |j'|^2) / rho),  D = rho - 1.
// The odd part 3 w c.j' then carries the momentum exactly as summed, instead of through
// the rounded u = j' / rho; the second-order part and the Guo term use 1 / rho.
//
// FP32 lattice constants: the collision conserves mass and momentum through two lattice
// identities, sum_i w_i = 1 (for w_i D) and sum_i 3 w_i c_ix^2 = 1 (for the odd part
// 3 w_i c_i.j'). With 1/3, 1/18, 1/36 rounded to FP32 the second is off by 3.0e-8, so
// every collision would add 3e-8 omega j' of momentum: a force proportional to the local
// velocity, a relative velocity error of ~3e-8 omega u / F in a slow steady flow. These
// constants satisfy both identities exactly in binary arithmetic (w1 = 14913080 2^-28,
// w2 = w1 / 2, w0 = 1 - 6 w1 - 12 w2 = 11184812 2^-25; a_k replaces 3 w_k in the odd
// part with 2 a1 + 8 a2 = 1: a1 = 11184810 2^-26, a2 = 11184811 2^-27) and differ from
// the exact weights by less than 2e-7 relative.
constexpr float W0S = 11184812.0f / 33554432.0f;
constexpr float W1S = 14913080.0f / 268435456.0f;
constexpr float W2S = 7456540.0f / 268435456.0f;
constexpr float A1S = 11184810.0f / 67108864.0f;
constexpr float A2S = 11184811.0f / 134217728.0f;

template <typename R>
__device__ __forceinline__ void bgk_pair_j(R& a, R& b, R w, R aw, R cj, R cF, R D, R inv_rho, R jj15, R uF3,
                                           R omega, R om1, R beta) {
    const R cu = cj * inv_rho;
    const R E = w * D + w * ((R(4.5) * cj * cj - jj15) * inv_rho);
    const R O = aw * cj;
    const R bw = beta * w;
    const R Se = bw * (R(9) * cu * cF - uF3);
    const R So = (beta * aw) * cF;
    a = om1 * a + (omega * (E + O) + (Se + So));
    b = om1 * b + (omega * (E - O) + (Se - So));
}

// Equilibrium of one direction pair: v_i = w (D + rho (3 cu + 4.5 cu^2 - 1.5 u.u)).
template <typename R>
__device__ __forceinline__ void eq_pair(R& a, R& b, R w, R cu, R D, R rho, R uu15) {
    const R E = w * D + (w * rho) * (R(4.5) * cu * cu - uu15);
    const R O = R(3) * (w * rho) * cu;
    a = E + O;
    b = E - O;
}

// One node's collision, in place on v[19].
template <typename R, bool SHIFT>
__device__ __forceinline__ void collide(R v[Q], int type, const StepParams& p, R Fx, R Fy, R Fz) {
    // moments from pair sums s and differences d of opposite directions
    const R s13 = v[1] + v[3], s24 = v[2] + v[4], s56 = v[5] + v[6], s79 = v[7] + v[9], s810 = v[8] + v[10];
    const R s1114 = v[11] + v[14], s1213 = v[12] + v[13], s1518 = v[15] + v[18], s1617 = v[16] + v[17];
    const R d13 = v[1] - v[3], d24 = v[2] - v[4], d56 = v[5] - v[6], d79 = v[7] - v[9], d810 = v[8] - v[10];
    const R d1114 = v[11] - v[14], d1213 = v[12] - v[13], d1518 = v[15] - v[18], d1617 = v[16] - v[17];
    const R sum = ((v[0] + s13) + (s24 + s56)) + ((s79 + s810) + (s1114 + s1213)) + (s1518 + s1617);
    const R jx = ((d13 + d79) - d810) + (d1114 + d1213);
    const R jy = ((d24 + d79) + d810) + (d1518 + d1617);
    const R jz = ((d56 + d1114) - d1213) + (d1518 - d1617);
    R D, rho;
    if (SHIFT) {
        D = sum;
        rho = R(1) + D;
    } else {
        rho = sum;
        D = sum;
    }
    const R inv_rho = R(1) / rho;
    const R Jx = jx + R(0.5) * Fx, Jy = jy + R(0.5) * Fy, Jz = jz + R(0.5) * Fz;
    const R ux = Jx * inv_rho;
    const R uy = Jy * inv_rho;
    const R uz = Jz * inv_rho;
    const R w0 = R(wgt(0)), w1 = R(wgt(1)), w2 = R(wgt(7));
    if (SHIFT && type == LBM_FLUID) {
        const R omega = par<R>(p.omega, p.omega_f), om1 = R(1) - omega, beta = par<R>(p.beta, p.beta_f);
        const R jj15 = R(1.5) * (Jx * Jx + Jy * Jy + Jz * Jz);
        const R uF3 = R(3) * (ux * Fx + uy * Fy + uz * Fz);
        const R s0 = R(W0S), s1 = R(W1S), s2 = R(W2S), a1 = R(A1S), a2 = R(A2S);
        v[0] = om1 * v[0] + (omega * (s0 * D - s0 * (jj15 * inv_rho)) - (beta * s0) * uF3);
        bgk_pair_j(v[1], v[3], s1, a1, Jx, Fx, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[2], v[4], s1, a1, Jy, Fy, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[5], v[6], s1, a1, Jz, Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[7], v[9], s2, a2, Jx + Jy, Fx + Fy, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[8], v[10], s2, a2, Jy - Jx, Fy - Fx, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[11], v[14], s2, a2, Jx + Jz, Fx + Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[12], v[13], s2, a2, Jx - Jz, Fx - Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[15], v[18], s2, a2, Jy + Jz, Fy + Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[16], v[17], s2, a2, Jy - Jz, Fy - Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
    } else if (type == LBM_FLUID) {
        const R omega = par<R>(p.omega, p.omega_f), om1 = R(1) - omega, beta = par<R>(p.beta, p.beta_f);
        const R uu15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
        const R uF3 = R(3) * (ux * Fx + uy * Fy + uz * Fz);
        v[0] = om1 * v[0] + (omega * (w0 * D - (w0 * rho) * uu15) - (beta * w0) * uF3);
        bgk_pair(v[1], v[3], w1, ux, Fx, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[2], v[4], w1, uy, Fy, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[5], v[6], w1, uz, Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[7], v[9], w2, ux + uy, Fx + Fy, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[8], v[10], w2, uy - ux, Fy - Fx, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[11], v[14], w2, ux + uz, Fx + Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[12], v[13], w2, ux - uz, Fx - Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[15], v[18], w2, uy + uz, Fy + Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[16], v[17], w2, uy - uz, Fy - Fz, D, rho, uu15, uF3, omega, om1, beta);
    } else {
        // inlet: f^eq(rho, u_in); outlet: f^eq(rho_out, u)
        R ex, ey, ez, Dq, rq;
        if (type == LBM_INLET) {
            ex = par<R>(p.u_in[0], p.u_in_f[0]);
            ey = par<R>(p.u_in[1], p.u_in_f[1]);
            ez = par<R>(p.u_in[2], p.u_in_f[2]);
            Dq = D; rq = rho;
        } else {
            ex = ux; ey = uy; ez = uz;
            rq = par<R>(p.rho_out, p.rho_out_f);
            Dq = SHIFT ? par<R>(p.rho_out - 1.0, p.rho_out_m1_f) : rq;
        }
        const R uu15 = R(1.5) * (ex * ex + ey * ey + ez * ez);
        v[0] = w0 * Dq - (w0 * rq) * uu15;
        eq_pair(v[1], v[3], w1, ex, Dq, rq, uu15);
        eq_pair(v[2], v[4], w1, ey, Dq, rq, uu15);
        eq_pair(v[5], v[6], w1, ez, Dq, rq, uu15);
        eq_pair(v[7], v[9], w2, ex + ey, Dq, rq, uu15);
        eq_pair(v[8], v[10], w2, ey - ex, Dq, rq, uu15);
        eq_pair(v[11], v[14], w2, ex + ez, Dq, rq, uu15);
        eq_pair(v[12], v[13], w2, ex - ez, Dq, rq, uu15);
        eq_pair(v[15], v[18], w2, ey + ez, Dq, rq, uu15);
        eq_pair(v[16], v[17], w2, ey - ez, Dq, rq, uu15);
    }
}

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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Staged element: the stored element for F64/F32; for F16S the aligned 32-bit word that
// holds the wanted half (cp.async moves at least 4 bytes), with the half picked later.
template <int DT> struct Staged { using E = uint32_t; };
template <> struct Staged<LBM_F64> { using E = uint64_t; };

template <int DT>
struct StepSmem {
    using E = typename Staged<DT>::E;
    using G = typename Store<DT>::R;
    int4 hdr[HDR_SLOTS];                                   // {t0, tiles, f0, nodes}
    int32_t nbr[META_SLOTS][GROUP_MAX_TILES][NBR_STRIDE];
    uint32_t word[META_SLOTS][STEP_THREADS];
    G gf[META_SLOTS][STEP_THREADS];
    E data[DATA_SLOTS][Q][STEP_THREADS];
};

__device__ __forceinline__ void issue_hdr(int4* hdr, int64_t grp, int64_t n_groups, const int4* __restrict__ groups) {
    if (threadIdx.x == 0 && grp < n_groups) cp_async16(hdr, groups + grp);
}

// Neighbour records of the group's tiles, and the words (and forces) of its nodes.
template <int DT>
__device__ __forceinline__ void issue_meta(StepSmem<DT>& sm, int mslot, const int4 h, const int32_t* __restrict__ nbr,
                                           const uint32_t* __restrict__ fword, const void* gfield_c) {
    const int t = threadIdx.x;
    if (t < h.y * (NBR_STRIDE / 4)) {
        const int lt = t / (NBR_STRIDE / 4), c = t % (NBR_STRIDE / 4);
        cp_async16(&sm.nbr[mslot][lt][4 * c], nbr + (int64_t)(h.x + lt) * NBR_STRIDE + 4 * c);
    }
    if (t < h.w) {
        cp_async4(&sm.word[mslot][t], fword + h.z + t);
        if (gfield_c) {
            const typename Store<DT>::R* g = static_cast<const typename Store<DT>::R*>(gfield_c);
            if (DT == LBM_F64) cp_async8(&sm.gf[mslot][t], g + h.z + t);
            else cp_async4(&sm.gf[mslot][t], g + h.z + t);
        }
    } else {
        sm.word[mslot][t] = 0;   // no node: idle thread
    }
}

// Issue the 19 gathers of this thread's node. Returns, for F16S, the mask of directions
// whose half is the upper half of the staged word.
template <int DT, int MODE>
__device__ __forceinline__ uint32_t issue_gather(StepSmem<DT>& sm, int mslot, int dslot, const int4 h,
                                                 const typename Store<DT>::T* __restrict__ A) {
    using T = typename Store<DT>::T;
    const int t = threadIdx.x;
    const uint32_t w = sm.word[mslot][t];
    uint32_t odd = 0;
    if (((w >> WORD_TYPE_SHIFT) & 3u) == LBM_SOLID) return 0;
    const int lt = (int)((w >> WORD_LT_SHIFT) & 7u), s = (int)((w >> WORD_SLOT_SHIFT) & 63u);
    const int x = s & 3, y = (s >> 2) & 3, z = s >> 4;
    const int64_t own = (int64_t)(h.x + lt) * (Q * SLOTS);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        int64_t src;
        if (MODE == STEP_RW) {
            src = own + i * SLOTS + s;   // read/write only: the node's own values
        } else if ((w >> i) & 1) {
            src = own + inv(i) * SLOTS + s;
        } else {
            const int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);
            const int nb = 13 + (sx >> 2) + 3 * (sy >> 2) + 9 * (sz >> 2);
            const int ss = (sx & 3) | ((sy & 3) << 2) | ((sz & 3) << 4);
            src = (int64_t)sm.nbr[mslot][lt][nb] * (Q * SLOTS) + i * SLOTS + ss;
        }
        if (DT == LBM_F64) {
            cp_async8(&sm.data[dslot][i][t], A + src);
        } else if (DT == LBM_F32) {
            cp_async4(&sm.data[dslot][i][t], A + src);
        } else {
            odd |= (uint32_t)(src & 1) << i;
            cp_async4(&sm.data[dslot][i][t], reinterpret_cast<const char*>(A) + (src & ~(int64_t)1) * sizeof(T));
        }
    }
    return odd;
}

// ------------------------------------------------------------ stochastic rounding
// MurmurHash3's 32-bit finaliser (A. Appleby, public domain): a bijective avalanche mix,
// used as a counter-based generator keyed by (step counter, node, direction pair).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// binary16 nearest to x + d, d = (r - 32767.5) 2^-16 s uniform over one binary16 spacing
// s of x (r: 16 random bits). For x in (lo, lo + s) this rounds up with probability
// (x - lo) / s to 16 bits, i.e. stochastic rounding (the FP32 sum x + d is off by at most
// 2^-14 s). s = 2^(e - 10) for |x| >= 2^-14 (e the exponent of x), 2^-24 below.
__device__ __forceinline__ __half half_dithered(float x, uint32_t r) {
    const uint32_t eb = __float_as_uint(x) & 0x7f800000u;
    const uint32_t sb = max(eb, 113u << 23) - (26u << 23);   // s * 2^-16
    const float d = __fmul_rn(__int2float_rn((int)r - 32767) - 0.5f, __uint_as_float(sb));
    return __float2half_rn(__fadd_rn(x, d));
}

template <int DT, bool VAR, int MODE>
__device__ __forceinline__ void compute_store(StepSmem<DT>& sm, int mslot, int dslot, const int4 h, uint32_t odd,
                                              typename Store<DT>::T* __restrict__ B, const StepParams& p,
                                              bool has_gf, uint32_t key) {
    using R = typename Store<DT>::R;
    using T = typename Store<DT>::T;
    const int t = threadIdx.x;
    const uint32_t w = sm.word[mslot][t];
    const int type = (int)((w >> WORD_TYPE_SHIFT) & 3u);
    if (type == LBM_SOLID) return;
    const int lt = (int)((w >> WORD_LT_SHIFT) & 7u), s = (int)((w >> WORD_SLOT_SHIFT) & 63u);
    R v[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        T e;
        if (DT == LBM_F16S) {
            const uint32_t word = (uint32_t)sm.data[dslot][i][t];
            const unsigned short hbits = (unsigned short)(((odd >> i) & 1) ? (word >> 16) : (word & 0xffffu));
            e = *reinterpret_cast<const T*>(&hbits);
        } else {
            const typename Staged<DT>::E raw = sm.data[dslot][i][t];
            e = *reinterpret_cast<const T*>(&raw);
        }
        v[i] = to_arith<DT>(e, i);
    }
    const R Fx = has_gf ? sm.gf[mslot][t] : par<R>(p.g[0], p.g_f[0]);
    const R Fy = par<R>(p.g[1], p.g_f[1]), Fz = par<R>(p.g[2], p.g_f[2]);
    if constexpr (MODE != STEP_FULL) {
        // calibration kernels: no collision, the gathered values are stored as they are
    } else if constexpr (DT == LBM_F64 && !VAR) {
        // FP64 storage: double-float collision for fluid nodes, FP64 for the closures
        if (type == LBM_FLUID) collide_df(v, (double)Fx, p.dfc);
        else collide<R, false>(v, type, p, Fx, Fy, Fz);
    } else {
        collide<R, Store<DT>::SHIFT>(v, type, p, Fx, Fy, Fz);
    }
    const int64_t own = (int64_t)(h.x + lt) * (Q * SLOTS);
    if constexpr (DT == LBM_F16S && VAR && MODE == STEP_FULL) {
        // stochastic rounding: two 16-bit dithers per hash of (key, node, pair)
        const uint32_t node = fmix32(key ^ (uint32_t)((h.x + lt) * SLOTS + s));
#pragma unroll
        for (int i = 0; i < Q; i += 2) {
            const uint32_t r = fmix32(node + (uint32_t)(i >> 1) * 0x9e3779b9u);
            B[own + i * SLOTS + s] = half_dithered(v[i] * F16_SCALE, r & 0xffffu);
            if (i + 1 < Q) B[own + (i + 1) * SLOTS + s] = half_dithered(v[i + 1] * F16_SCALE, r >> 16);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) B[own + i * SLOTS + s] = to_store<DT>(v[i], i);
    }
}

// Resident CTAs per SM the kernel is compiled for: shared memory allows 4 CTAs of the
// 4-byte formats (about 46 KB each) and 2 of FP64 (about 88 KB each); registers match.
template <int DT> struct StepOcc { static constexpr int CTAS = 4; };
template <> struct StepOcc<LBM_F64> { static constexpr int CTAS = 2; };

template <int DT, bool VAR, int MODE>
__global__ void __launch_bounds__(STEP_THREADS, StepOcc<DT>::CTAS)
k_step(const typename Store<DT>::T* __restrict__ A, typename Store<DT>::T* __restrict__ B,
       const int4* __restrict__ groups, const int32_t* __restrict__ nbr, const uint32_t* __restrict__ fword,
       const void* __restrict__ gfield_c, int64_t n_groups, StepParams p, const uint32_t* __restrict__ seed_in,
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
    issue_meta<DT>(sm, 0, sm.hdr[0], nbr, fword, gfield_c);
    cp_async_commit();
    if (g0 + G < n_groups) issue_meta<DT>(sm, 1, sm.hdr[1], nbr, fword, gfield_c);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    uint32_t odd_cur = issue_gather<DT, MODE>(sm, 0, 0, sm.hdr[0], A);
    cp_async_commit();
    int it = 0;
    for (int64_t g = g0; g < n_groups; g += G, it++) {
        // pending: header(g + 2G) [done], meta(g + G), gather(g)
        cp_async_wait<1>();
        __syncthreads();   // header(g + 2G), meta(g + G) visible; iteration it - 1 finished
        issue_hdr(&sm.hdr[(it + 3) & 3], g + 3 * G, n_groups, groups);
        cp_async_commit();
        if (g + 2 * G < n_groups) issue_meta<DT>(sm, (it + 2) % META_SLOTS, sm.hdr[(it + 2) & 3], nbr, fword, gfield_c);
        cp_async_commit();
        uint32_t odd_next = 0;
        if (g + G < n_groups)
            odd_next = issue_gather<DT, MODE>(sm, (it + 1) % META_SLOTS, (it + 1) & 1, sm.hdr[(it + 1) & 3], A);
        cp_async_commit();
        // pending: gather(g), header(g + 3G), meta(g + 2G), gather(g + G)
        cp_async_wait<3>();
        compute_store<DT, VAR, MODE>(sm, it % META_SLOTS, it & 1, sm.hdr[it & 3], odd_cur, B, p, has_gf, key);
        odd_cur = odd_next;
    }
    cp_async_wait<0>();
}

template <int DT, bool VAR, int MODE>
static int step_grid(int64_t n_groups) {
    static int per_sm = -1, n_sm = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_step<DT, VAR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(StepSmem<DT>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<DT, VAR, MODE>, STEP_THREADS,
                                                      sizeof(StepSmem<DT>));
        if (per_sm < 1) per_sm = 1;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(n_groups, (int64_t)per_sm * n_sm));
}

template <int DT, bool VAR, int MODE>
static cudaError_t launch_step_dt(lbm_ctx* c, const void* A, void* B) {
    using T = typename Store<DT>::T;
    const int grid = step_grid<DT, VAR, MODE>(c->n_groups);
    // the copy read decides which counter is read and which is advanced
    const int from = A == c->f[0] ? 0 : 1;
    const uint32_t* seed_in = c->seed ? c->seed + from : nullptr;
    uint32_t* seed_out = c->seed ? c->seed + (1 - from) : nullptr;
    k_step<DT, VAR, MODE><<<grid, STEP_THREADS, sizeof(StepSmem<DT>), c->stream>>>(
        (const T*)A, (T*)B, c->groups, c->nbr, c->fword, c->gfield ? c->gfield_c : nullptr, c->n_groups, c->p,
        seed_in, seed_out);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_step_mode(lbm_ctx* c, const void* A, void* B) {
    switch (c->dtype) {
        case LBM_F64:
            return c->native64 ? launch_step_dt<LBM_F64, true, MODE>(c, A, B)
                               : launch_step_dt<LBM_F64, false, MODE>(c, A, B);
        case LBM_F32: return launch_step_dt<LBM_F32, false, MODE>(c, A, B);
        default:
            return c->sr ? launch_step_dt<LBM_F16S, true, MODE>(c, A, B)
                         : launch_step_dt<LBM_F16S, false, MODE>(c, A, B);
    }
}

cudaError_t launch_step(lbm_ctx* c, const void* A, void* B) { return launch_step_kind(c, STEP_FULL, A, B); }

// One-time kernel attributes and occupancy query of the fused step, done outside any
// stream capture.
cudaError_t prepare_step(lbm_ctx* c) {
    switch (c->dtype) {
        case LBM_F64:
            if (c->native64) step_grid<LBM_F64, true, STEP_FULL>(1);
            else step_grid<LBM_F64, false, STEP_FULL>(1);
            break;
        case LBM_F32: step_grid<LBM_F32, false, STEP_FULL>(1); break;
        default:
            if (c->sr) step_grid<LBM_F16S, true, STEP_FULL>(1);
            else step_grid<LBM_F16S, false, STEP_FULL>(1);
    }
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
