// lbm_step.cu -- the fused collide-and-stream step kernel (Sec. 3.4, Algorithm 2).
//
// One CTA of 128 threads handles two kept tiles; thread s of a tile owns slot s
// (node x + 4 y + 16 z of the tile). Per CTA:
//   1. stage the 3x3x3 neighbourhood of each tile (tile ranks -> element offsets of the
//      tile's data blocks) and the neighbours' 64-bit solid masks in shared memory
//      (the local tileMap / nodeType copies of Algorithm 2, as bit masks), one barrier;
//   2. every non-solid node pulls f_i from x - c_i: from its own tile or a neighbour
//      tile's data block i; a solid, dropped or out-of-box source gives halfway
//      bounce-back f_i(x) <- A_inv(i)(x) (Sec. 2.2 walls; propagation only between
//      non-solid nodes, Sec. 3.4);
//   3. moments, boundary closures (inlet / outlet) or LBGK + Guo collision (Eq. 2, 3, 7);
//   4. store all 19 populations to the other copy, coalesced (64 consecutive slots of a
//      data block per warp pair).
// Solid nodes issue no loads and no stores. All 19 gathers of a thread are independent
// loads, so each thread keeps 19 requests in flight.
#include <algorithm>

#include "lbm_internal.cuh"
#include "lbm_store.cuh"

namespace lbm {

constexpr int STEP_TILES = 2;
constexpr int STEP_THREADS = STEP_TILES * SLOTS;

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

template <int DT>
__global__ void __launch_bounds__(STEP_THREADS)
k_step(const typename Store<DT>::T* __restrict__ A, typename Store<DT>::T* __restrict__ B,
       const int32_t* __restrict__ nbr, const uint64_t* __restrict__ smask,
       const uint32_t* __restrict__ tflags, const uint8_t* __restrict__ ntype, int64_t n_tiles,
       StepParams p) {
    using R = typename Store<DT>::R;
    __shared__ int64_t s_base[STEP_TILES][NBR];   // element offset of a neighbour's block 0, -1 if absent
    __shared__ uint64_t s_mask[STEP_TILES][NBR];
    __shared__ uint32_t s_flag[STEP_TILES];
    const int lt = threadIdx.x >> 6;
    const int s = threadIdx.x & 63;
    const int64_t k = (int64_t)blockIdx.x * STEP_TILES + lt;
    if (s < NBR) {
        const int64_t nk = k < n_tiles ? (int64_t)nbr[k * NBR + s] : -1;
        s_base[lt][s] = nk >= 0 ? nk * (Q * SLOTS) : -1;
        s_mask[lt][s] = nk >= 0 ? smask[nk] : ~0ull;
    } else if (s == 32) {
        s_flag[lt] = k < n_tiles ? tflags[k] : 0u;
    }
    __syncthreads();
    if (k >= n_tiles) return;
    if ((s_mask[lt][13] >> s) & 1) return;   // solid node: no load, no store

    const int x = s & 3, y = (s >> 2) & 3, z = s >> 4;
    const int64_t own = k * (Q * SLOTS);
    R v[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);   // in [-1, 4]
        const int nb = 13 + (sx >> 2) + 3 * (sy >> 2) + 9 * (sz >> 2);
        const int ss = (sx & 3) | ((sy & 3) << 2) | ((sz & 3) << 4);
        const int64_t base = s_base[lt][nb];
        const bool bounce = base < 0 || ((s_mask[lt][nb] >> ss) & 1);
        const int64_t src = bounce ? own + inv(i) * SLOTS + s : base + i * SLOTS + ss;
        v[i] = to_arith<DT>(A[src], i);
    }
    const int type = (s_flag[lt] & FLAG_HAS_BC) ? (int)ntype[k * SLOTS + s] : LBM_FLUID;
    const R Fx = p.gfield ? (R)gfield_at<DT>(p.gfield, k * SLOTS + s) : R(p.g[0]);
    collide<R, Store<DT>::SHIFT>(v, type, p, Fx, R(p.g[1]), R(p.g[2]));
#pragma unroll
    for (int i = 0; i < Q; i++) B[own + i * SLOTS + s] = to_store<DT>(v[i], i);
}

cudaError_t launch_step(lbm_ctx* c, const void* A, void* B) {
    if (c->n_tiles == 0) return cudaSuccess;
    const int64_t blocks = (c->n_tiles + STEP_TILES - 1) / STEP_TILES;
    switch (c->dtype) {
        case LBM_F64:
            k_step<LBM_F64><<<(unsigned)blocks, STEP_THREADS, 0, c->stream>>>(
                (const double*)A, (double*)B, c->nbr, c->smask, c->tflags, c->ntype, c->n_tiles, c->p);
            break;
        case LBM_F32:
            k_step<LBM_F32><<<(unsigned)blocks, STEP_THREADS, 0, c->stream>>>(
                (const float*)A, (float*)B, c->nbr, c->smask, c->tflags, c->ntype, c->n_tiles, c->p);
            break;
        default:
            k_step<LBM_F16S><<<(unsigned)blocks, STEP_THREADS, 0, c->stream>>>(
                (const __half*)A, (__half*)B, c->nbr, c->smask, c->tflags, c->ntype, c->n_tiles, c->p);
    }
    return cudaGetLastError();
}

}  // namespace lbm
