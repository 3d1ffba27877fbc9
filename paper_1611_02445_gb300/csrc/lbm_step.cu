// lbm_step.cu -- the fused collide-and-stream step kernel (Sec. 3.4, Algorithm 2).
//
// Work unit: a group of GROUP_TILES = 4 kept tiles, one thread per slot (256 threads;
// thread s of a tile owns node x + 4 y + 16 z). Persistent CTAs walk the groups
// b, b + G, b + 2G, ... with a software pipeline, so that while a group is computed the
// next group's gathers are already in flight:
//   meta(g)   cp.async of the group's neighbour records (the local tileMap copy of
//             Algorithm 2, 28 ranks per tile) and per-node gather words (which
//             directions bounce, node type) into a 3-slot shared-memory ring;
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

constexpr int GROUP_TILES = 4;
constexpr int STEP_THREADS = GROUP_TILES * SLOTS;   // 256
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
    const R sum = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) +
                  ((v[8] + v[9]) + (v[10] + v[11])) + ((v[12] + v[13]) + (v[14] + v[15])) +
                  ((v[16] + v[17]) + v[18]);
    const R jx = ((v[1] + v[7]) + (v[10] + v[11]) + v[12]) - ((v[3] + v[8]) + (v[9] + v[13]) + v[14]);
    const R jy = ((v[2] + v[7]) + (v[8] + v[15]) + v[16]) - ((v[4] + v[9]) + (v[10] + v[17]) + v[18]);
    const R jz = ((v[5] + v[11]) + (v[13] + v[15]) + v[17]) - ((v[6] + v[12]) + (v[14] + v[16]) + v[18]);
    R D, rho;
    if (SHIFT) {
        D = sum + R(WF_BIAS);
        rho = R(1) + D;
    } else {
        rho = sum;
        D = sum;
    }
    const R inv_rho = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * inv_rho;
    const R uy = (jy + R(0.5) * Fy) * inv_rho;
    const R uz = (jz + R(0.5) * Fz) * inv_rho;
    const R w0 = R(wgt(0)), w1 = R(wgt(1)), w2 = R(wgt(7));
    if (type == LBM_FLUID) {
        const R omega = R(p.omega), om1 = R(1) - omega, beta = R(p.beta);
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
            ex = R(p.u_in[0]); ey = R(p.u_in[1]); ez = R(p.u_in[2]);
            Dq = D; rq = rho;
        } else {
            ex = ux; ey = uy; ez = uz;
            rq = R(p.rho_out);
            Dq = SHIFT ? R(p.rho_out - 1.0) : rq;
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
    int32_t nbr[META_SLOTS][GROUP_TILES][NBR_STRIDE];
    uint32_t word[META_SLOTS][STEP_THREADS];
    G gf[META_SLOTS][STEP_THREADS];
    E data[DATA_SLOTS][Q][STEP_THREADS];
};

template <int DT>
__device__ __forceinline__ void issue_meta(StepSmem<DT>& sm, int slot, int64_t grp, int64_t n_tiles,
                                           const int32_t* __restrict__ nbr, const uint32_t* __restrict__ nword,
                                           const void* gfield) {
    const int t = threadIdx.x;
    const int64_t k0 = grp * GROUP_TILES;
    // neighbour records: GROUP_TILES x 112 bytes = 28 chunks of 16 bytes
    if (t < GROUP_TILES * (NBR_STRIDE / 4)) {
        const int lt = t / (NBR_STRIDE / 4), c = t % (NBR_STRIDE / 4);
        if (k0 + lt < n_tiles) cp_async16(&sm.nbr[slot][lt][4 * c], nbr + (k0 + lt) * NBR_STRIDE + 4 * c);
    }
    const int64_t k = k0 + (t >> 6);
    if (k < n_tiles) {
        cp_async4(&sm.word[slot][t], nword + k * SLOTS + (t & 63));
        if (gfield) {
            const typename Store<DT>::R* g = static_cast<const typename Store<DT>::R*>(gfield);
            if (DT == LBM_F64) cp_async8(&sm.gf[slot][t], g + k * SLOTS + (t & 63));
            else cp_async4(&sm.gf[slot][t], g + k * SLOTS + (t & 63));
        }
    } else {
        sm.word[slot][t] = 0;   // past the last tile: treated as solid
    }
}

// Issue the 19 gathers of this thread's node of group grp. Returns, for F16S, the mask
// of directions whose half is the upper half of the staged word.
template <int DT>
__device__ __forceinline__ uint32_t issue_gather(StepSmem<DT>& sm, int mslot, int dslot, int64_t grp,
                                                 const typename Store<DT>::T* __restrict__ A) {
    using T = typename Store<DT>::T;
    const int t = threadIdx.x, lt = t >> 6, s = t & 63;
    const uint32_t w = sm.word[mslot][t];
    uint32_t odd = 0;
    if ((w >> WORD_TYPE_SHIFT) == LBM_SOLID) return 0;
    const int x = s & 3, y = (s >> 2) & 3, z = s >> 4;
    const int64_t own = (grp * GROUP_TILES + lt) * (Q * SLOTS);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        int64_t src;
        if ((w >> i) & 1) {
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

template <int DT>
__device__ __forceinline__ void compute_store(StepSmem<DT>& sm, int mslot, int dslot, int64_t grp, uint32_t odd,
                                              typename Store<DT>::T* __restrict__ B, const StepParams& p) {
    using R = typename Store<DT>::R;
    using T = typename Store<DT>::T;
    const int t = threadIdx.x, lt = t >> 6, s = t & 63;
    const uint32_t w = sm.word[mslot][t];
    const int type = (int)(w >> WORD_TYPE_SHIFT);
    if (type == LBM_SOLID) return;
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
    const R Fx = p.gfield ? sm.gf[mslot][t] : R(p.g[0]);
    collide<R, Store<DT>::SHIFT>(v, type, p, Fx, R(p.g[1]), R(p.g[2]));
    const int64_t own = (grp * GROUP_TILES + lt) * (Q * SLOTS);
#pragma unroll
    for (int i = 0; i < Q; i++) B[own + i * SLOTS + s] = to_store<DT>(v[i], i);
}

// Resident CTAs per SM the kernel is compiled for: shared memory allows 4 CTAs of the
// 4-byte formats (46 KB each) and 2 of FP64 (88 KB each); registers are capped to match.
template <int DT> struct StepOcc { static constexpr int CTAS = 4; };
template <> struct StepOcc<LBM_F64> { static constexpr int CTAS = 2; };

template <int DT>
__global__ void __launch_bounds__(STEP_THREADS, StepOcc<DT>::CTAS)
k_step(const typename Store<DT>::T* __restrict__ A, typename Store<DT>::T* __restrict__ B,
       const int32_t* __restrict__ nbr, const uint32_t* __restrict__ nword, int64_t n_tiles,
       int64_t n_groups, StepParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepSmem<DT>& sm = *reinterpret_cast<StepSmem<DT>*>(smem_raw);
    const int64_t G = gridDim.x;
    const int64_t g0 = blockIdx.x;
    if (g0 >= n_groups) return;
    // prologue: meta(g0), meta(g0 + G), then gather(g0)
    issue_meta<DT>(sm, 0, g0, n_tiles, nbr, nword, p.gfield);
    cp_async_commit();
    if (g0 + G < n_groups) issue_meta<DT>(sm, 1, g0 + G, n_tiles, nbr, nword, p.gfield);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    uint32_t odd_cur = issue_gather<DT>(sm, 0, 0, g0, A);
    cp_async_commit();
    int it = 0;
    for (int64_t g = g0; g < n_groups; g += G, it++) {
        const int m_cur = it % META_SLOTS, m_next = (it + 1) % META_SLOTS, m_next2 = (it + 2) % META_SLOTS;
        const int d_cur = it & 1, d_next = (it + 1) & 1;
        // pending: meta(g + G), gather(g)
        cp_async_wait<1>();
        __syncthreads();   // meta(g + G) visible; everyone done with iteration it - 1
        if (g + 2 * G < n_groups) issue_meta<DT>(sm, m_next2, g + 2 * G, n_tiles, nbr, nword, p.gfield);
        cp_async_commit();
        uint32_t odd_next = 0;
        if (g + G < n_groups) odd_next = issue_gather<DT>(sm, m_next, d_next, g + G, A);
        cp_async_commit();
        // pending: gather(g), meta(g + 2G), gather(g + G)
        cp_async_wait<2>();
        compute_store<DT>(sm, m_cur, d_cur, g, odd_cur, B, p);
        odd_cur = odd_next;
    }
    cp_async_wait<0>();
}

template <int DT>
static int step_grid(int64_t n_groups) {
    static int per_sm = -1, n_sm = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_step<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(StepSmem<DT>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<DT>, STEP_THREADS, sizeof(StepSmem<DT>));
        if (per_sm < 1) per_sm = 1;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(n_groups, (int64_t)per_sm * n_sm));
}

template <int DT>
static cudaError_t launch_step_dt(lbm_ctx* c, const void* A, void* B) {
    using T = typename Store<DT>::T;
    const int64_t n_groups = (c->n_tiles + GROUP_TILES - 1) / GROUP_TILES;
    const int grid = step_grid<DT>(n_groups);
    k_step<DT><<<grid, STEP_THREADS, sizeof(StepSmem<DT>), c->stream>>>(
        (const T*)A, (T*)B, c->nbr, c->nword, c->n_tiles, n_groups, c->p);
    return cudaGetLastError();
}

cudaError_t launch_step(lbm_ctx* c, const void* A, void* B) {
    if (c->n_tiles == 0) return cudaSuccess;
    switch (c->dtype) {
        case LBM_F64: return launch_step_dt<LBM_F64>(c, A, B);
        case LBM_F32: return launch_step_dt<LBM_F32>(c, A, B);
        default: return launch_step_dt<LBM_F16S>(c, A, B);
    }
}

}  // namespace lbm
