// lbm_adjoint.cu -- discrete adjoint of the fused step, with checkpoint and recompute.
//
// The paper has no adjoint. Forward map of one step: s_{t+1} = C(G s_t), where G is the
// gather with halfway bounce-back (a permutation of (direction, node) slots) and C the
// node-local collision. For a loss L(s_T):
//   lambda_T = dL/ds_T,
//   mu_t     = J_C(G s_t)^T lambda_{t+1}          (node-local),
//   lambda_t = G^T mu_t: lambda_k(x) = mu_k(x + c_k) if x + c_k is not solid, else
//              mu_inv(k)(x)   (the transpose of the bounce-back permutation),
// and dL/dF(x), dL/dtau accumulate (dC/dF)^T lambda and (dC/dtau)^T lambda.
// One adjoint kernel per step reads s_t with the forward gather and mu_{t+1} with the
// transposed gather (both pull-shaped) and writes mu_t. Gradients accumulate in FP64:
// per node for F_x, per block for tau (each block always owns the same nodes, so the
// sums are deterministic).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lbm_internal.cuh"
#include "lbm_store.cuh"

namespace lbm {

constexpr int ADJ_THREADS = 128;
constexpr int LOSS_THREADS = 256;

template <int DT> using Arith = typename Store<DT>::R;

// Outlet-flux loss, pass 1: per-block sums of u_x and node counts over the non-solid
// nodes of the plane x = plane_x, u = (sum c f* - F/2)/rho from the stored populations.
template <int DT>
__global__ void __launch_bounds__(LOSS_THREADS) k_loss_partials(const typename Store<DT>::T* __restrict__ f,
                                                                const uint32_t* __restrict__ nword,
                                                                const uint32_t* __restrict__ non_empty,
                                                                const uint64_t* __restrict__ smask,
                                                                const int32_t* __restrict__ tlane,
                                                                const void* __restrict__ gfield, int64_t n_tiles,
                                                                int Tx, int plane_x, StepParams p,
                                                                double* __restrict__ partials) {
    double su = 0.0, cnt = 0.0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_tiles * SLOTS;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        if ((nword[idx] >> WORD_TYPE_SHIFT) == LBM_SOLID) continue;
        const int x = TILE * (int)(non_empty[k] % (uint32_t)Tx) + (s & 3);
        if (x != plane_x) continue;
        const uint32_t P = node_lane((uint32_t)tlane[k], smask[k], s);
        double r = 0.0, jx = 0.0;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const double v = to_f64<DT>(f[data_index(P, i)], i);
            r += v;
            jx += cx(i) * v;
        }
        const double Fx = gfield ? gfield_at<DT>(gfield, idx) : p.g[0];
        su += (jx - 0.5 * Fx) / r;
        cnt += 1.0;
    }
    __shared__ double sh[2][LOSS_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_down_sync(0xffffffffu, su, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        sh[0][warp] = su;
        sh[1][warp] = cnt;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < LOSS_THREADS / 32; w++) v += sh[threadIdx.x][w];
        partials[blockIdx.x * 2 + threadIdx.x] = v;
    }
}

// Fixed-order sum of per-block partials with `width` components each.
__global__ void k_sum_partials(const double* __restrict__ partials, int nb, int width, double* __restrict__ out) {
    if (threadIdx.x < width) {
        double v = 0.0;
        for (int b = 0; b < nb; b++) v += partials[b * width + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

// Seed of the reverse sweep: lambda_T = dL/df* = (c_x - u_x)/(rho |P|) on the plane, 0
// elsewhere; the direct term dL/dF_x = -1/(2 rho |P|) starts the per-node gradient.
template <int DT>
__global__ void k_loss_seed(const typename Store<DT>::T* __restrict__ f, const uint32_t* __restrict__ nword,
                            const uint32_t* __restrict__ non_empty, const uint64_t* __restrict__ smask,
                            const int32_t* __restrict__ tlane, const void* __restrict__ gfield,
                            int64_t n_tiles, int Tx, int plane_x, StepParams p, const double* __restrict__ sums,
                            Arith<DT>* __restrict__ lam, double* __restrict__ gbar) {
    using R = Arith<DT>;
    const double count = sums[1];
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_tiles * SLOTS;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const bool nonsolid = (nword[idx] >> WORD_TYPE_SHIFT) != LBM_SOLID;
        if (!nonsolid) continue;   // solid slots have no storage
        const uint32_t P = node_lane((uint32_t)tlane[k], smask[k], s);
        const bool on = TILE * (int)(non_empty[k] % (uint32_t)Tx) + (s & 3) == plane_x;
        double r = 1.0, ux = 0.0;
        if (on) {
            double jx = 0.0;
            r = 0.0;
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const double v = to_f64<DT>(f[data_index(P, i)], i);
                r += v;
                jx += cx(i) * v;
            }
            const double Fx = gfield ? gfield_at<DT>(gfield, idx) : p.g[0];
            ux = (jx - 0.5 * Fx) / r;
        }
#pragma unroll
        for (int i = 0; i < Q; i++) lam[data_index(P, i)] = on ? (R)((cx(i) - ux) / (r * count)) : R(0);
        gbar[idx] = on ? -0.5 / (r * count) : 0.0;
    }
}

// Transposed collision Jacobian at one node, in moment form. v: gathered populations
// (f, or h = f - w for the shifted formats), lam: adjoint of the post-collision values.
// Writes mu (adjoint of the gathered values), returns dL/dF_x and adds dL/dtau.
template <typename R, bool SHIFT>
__device__ __forceinline__ R collide_adjoint(const R v[Q], const R lam[Q], int type, const StepParams& p, R Fx, R Fy,
                                             R Fz, R mu[Q], double& taubar) {
    R sum = 0, jx = 0, jy = 0, jz = 0;
    R M0 = 0, M1x = 0, M1y = 0, M1z = 0, Mxx = 0, Myy = 0, Mzz = 0, Mxy = 0, Mxz = 0, Myz = 0, Lv = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        sum += v[i];
        jx += R(cx(i)) * v[i];
        jy += R(cy(i)) * v[i];
        jz += R(cz(i)) * v[i];
        const R wl = R(wgt(i)) * lam[i];
        M0 += wl;
        M1x += R(cx(i)) * wl;
        M1y += R(cy(i)) * wl;
        M1z += R(cz(i)) * wl;
        Mxx += R(cx(i) * cx(i)) * wl;
        Myy += R(cy(i) * cy(i)) * wl;
        Mzz += R(cz(i) * cz(i)) * wl;
        Mxy += R(cx(i) * cy(i)) * wl;
        Mxz += R(cx(i) * cz(i)) * wl;
        Myz += R(cy(i) * cz(i)) * wl;
        Lv += lam[i] * v[i];
    }
    R D, rho;
    if (SHIFT) {
        D = sum;
        rho = R(1) + D;
    } else {
        rho = sum;
        D = sum;
    }
    const R ux = (jx + R(0.5) * Fx) / rho, uy = (jy + R(0.5) * Fy) / rho, uz = (jz + R(0.5) * Fz) / rho;
    R rhobar = 0, ubx = 0, uby = 0, ubz = 0, Fbx = 0;
    R keep = 0;   // coefficient of lam_i kept in mu_i
    if (type == LBM_INLET) {
        const R ex = par<R>(p.u_in[0], p.u_in_f[0]), ey = par<R>(p.u_in[1], p.u_in_f[1]),
                ez = par<R>(p.u_in[2], p.u_in_f[2]);
        const R M2ex = Mxx * ex + Mxy * ey + Mxz * ez, M2ey = Mxy * ex + Myy * ey + Myz * ez,
                M2ez = Mxz * ex + Myz * ey + Mzz * ez;
        rhobar = M0 * (R(1) - R(1.5) * (ex * ex + ey * ey + ez * ez)) + R(3) * (M1x * ex + M1y * ey + M1z * ez) +
                 R(4.5) * (ex * M2ex + ey * M2ey + ez * M2ez);
#pragma unroll
        for (int i = 0; i < Q; i++) mu[i] = rhobar;
        return R(0);
    }
    const R M2ux = Mxx * ux + Mxy * uy + Mxz * uz, M2uy = Mxy * ux + Myy * uy + Myz * uz,
            M2uz = Mxz * ux + Myz * uy + Mzz * uz;
    if (type == LBM_OUTLET) {
        const R ro = par<R>(p.rho_out, p.rho_out_f);
        ubx = ro * (R(3) * M1x + R(9) * M2ux - R(3) * ux * M0);
        uby = ro * (R(3) * M1y + R(9) * M2uy - R(3) * uy * M0);
        ubz = ro * (R(3) * M1z + R(9) * M2uz - R(3) * uz * M0);
    } else {
        const R omega = par<R>(p.omega, p.omega_f), beta = par<R>(p.beta, p.beta_f);
        const R uu = ux * ux + uy * uy + uz * uz, uF = ux * Fx + uy * Fy + uz * Fz;
        const R M1u = M1x * ux + M1y * uy + M1z * uz, M1F = M1x * Fx + M1y * Fy + M1z * Fz;
        const R uM2u = ux * M2ux + uy * M2uy + uz * M2uz;
        const R M2Fx = Mxx * Fx + Mxy * Fy + Mxz * Fz, M2Fy = Mxy * Fx + Myy * Fy + Myz * Fz,
                M2Fz = Mxz * Fx + Myz * Fy + Mzz * Fz;
        const R uM2F = ux * M2Fx + uy * M2Fy + uz * M2Fz;
        const R P = R(3) * M1u + R(4.5) * uM2u - R(1.5) * uu * M0;   // sum w lam (e_i - 1)
        rhobar = omega * (M0 + P);
        ubx = omega * rho * (R(3) * M1x + R(9) * M2ux - R(3) * ux * M0) + beta * (R(9) * M2Fx - R(3) * Fx * M0);
        uby = omega * rho * (R(3) * M1y + R(9) * M2uy - R(3) * uy * M0) + beta * (R(9) * M2Fy - R(3) * Fy * M0);
        ubz = omega * rho * (R(3) * M1z + R(9) * M2uz - R(3) * uz * M0) + beta * (R(9) * M2Fz - R(3) * Fz * M0);
        Fbx = beta * (R(3) * M1x - R(3) * ux * M0 + R(9) * M2ux);
        // dL/dtau: sum lam (v - v^eq) / tau^2 + (1/(2 tau^2)) sum lam w Q
        const R lam_diff = Lv - (D * M0 + rho * P);
        const R lwq = R(3) * M1F - R(3) * uF * M0 + R(9) * uM2F;
        const double it2 = p.omega * p.omega;
        taubar += ((double)lam_diff + 0.5 * (double)lwq) * it2;
        keep = R(1) - omega;
    }
    const R ir = R(1) / rho;
    Fbx += R(0.5) * ubx * ir;
    rhobar -= (ubx * ux + uby * uy + ubz * uz) * ir;
    const R jbx = ubx * ir, jby = uby * ir, jbz = ubz * ir;
#pragma unroll
    for (int i = 0; i < Q; i++) mu[i] = keep * lam[i] + rhobar + R(cx(i)) * jbx + R(cy(i)) * jby + R(cz(i)) * jbz;
    return Fbx;
}

// One reverse step: mu_out = J_C(G s_t)^T lambda_{t+1}, lambda_{t+1} = G^T mu_in (or
// mu_in itself when direct, for the seed of the last step). One thread per non-solid
// node of the compact node list (the step kernel's per-node words and slot indices), so
// no lane idles on a solid slot; neighbour tile ranks come through the read-only cache.
// Block b always owns the nodes [b ADJ_THREADS, (b + 1) ADJ_THREADS): its dL/dtau
// partial is deterministic.
template <int DT>
__global__ void __launch_bounds__(ADJ_THREADS) k_adjoint(const typename Store<DT>::T* __restrict__ st,
                                                         const Arith<DT>* __restrict__ mu_in, int direct,
                                                         Arith<DT>* __restrict__ mu_out,
                                                         const int32_t* __restrict__ nbr,
                                                         const uint64_t* __restrict__ smask,
                                                         const int32_t* __restrict__ tlane,
                                                         const uint32_t* __restrict__ fword,
                                                         const uint32_t* __restrict__ fidx,
                                                         const void* __restrict__ gfield, int64_t n_nodes,
                                                         StepParams p, double* __restrict__ gbar,
                                                         double* __restrict__ tau_part) {
    using R = Arith<DT>;
    __shared__ double s_tau[ADJ_THREADS / 32];
    const int64_t n = (int64_t)blockIdx.x * ADJ_THREADS + threadIdx.x;
    double taubar = 0.0;
    if (n < n_nodes) {
        const uint32_t w = __ldg(fword + n);
        const uint32_t gi = __ldg(fidx + n);
        const int type = (int)((w >> WORD_TYPE_SHIFT) & 3u);
        const int64_t k = gi >> 6;
        const int s = (int)(gi & 63u);
        const int x = s & 3, y = (s >> 2) & 3, z = s >> 4;
        const uint32_t own = node_lane((uint32_t)__ldg(tlane + k), __ldg(smask + k), s);
        R v[Q], lam[Q], mu[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) {
            // forward gather of direction i and, with the same source, the transposed
            // gather of direction inv(i): lambda_inv(i)(x) = mu_inv(i)(x - c_i)
            const int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);
            const int nb = 13 + (sx >> 2) + 3 * (sy >> 2) + 9 * (sz >> 2);
            const int ss = (sx & 3) | ((sy & 3) << 2) | ((sz & 3) << 4);
            const bool bounce = (w >> i) & 1;
            uint32_t src = own;
            if (!bounce) {
                const int64_t r = nb == 13 ? k : (int64_t)__ldg(nbr + k * NBR_STRIDE + nb);
                src = node_lane((uint32_t)__ldg(tlane + r), __ldg(smask + r), ss);
            }
            v[i] = to_arith<DT>(st[data_index(src, bounce ? inv(i) : i)], i);
            if (direct) {
                lam[inv(i)] = mu_in[data_index(own, inv(i))];
            } else {
                lam[inv(i)] = mu_in[data_index(src, bounce ? i : inv(i))];
            }
        }
        const R Fx = gfield ? (R)gfield_at<DT>(gfield, (int64_t)gi) : par<R>(p.g[0], p.g_f[0]);
        const R Fb = collide_adjoint<R, Store<DT>::SHIFT>(v, lam, type, p, Fx, par<R>(p.g[1], p.g_f[1]),
                                                          par<R>(p.g[2], p.g_f[2]), mu, taubar);
#pragma unroll
        for (int i = 0; i < Q; i++) mu_out[data_index(own, i)] = mu[i];
        gbar[gi] += (double)Fb;
    }
    for (int o = 16; o > 0; o >>= 1) taubar += __shfl_down_sync(0xffffffffu, taubar, o);
    if ((threadIdx.x & 31) == 0) s_tau[threadIdx.x >> 5] = taubar;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < ADJ_THREADS / 32; i++) t += s_tau[i];
        tau_part[blockIdx.x] += t;
    }
}

// Tile-major per-node gradient -> dense array (zeroed by the caller).
__global__ void k_gbar_dense(const double* __restrict__ gbar, const uint32_t* __restrict__ nword,
                             const uint32_t* __restrict__ non_empty, int64_t n_tiles, int nx, int ny, int Tx,
                             int Ty, double* __restrict__ dense) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_tiles * SLOTS;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if ((nword[idx] >> WORD_TYPE_SHIFT) == LBM_SOLID) continue;
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const uint32_t t = non_empty[k];
        const int x = TILE * (int)(t % (uint32_t)Tx) + (s & 3);
        const int y = TILE * (int)((t / (uint32_t)Tx) % (uint32_t)Ty) + ((s >> 2) & 3);
        const int z = TILE * (int)(t / ((uint32_t)Tx * (uint32_t)Ty)) + (s >> 4);
        dense[x + (int64_t)nx * (y + (int64_t)ny * z)] = gbar[idx];
    }
}

namespace {

struct DevBuf {
    void* p = nullptr;
    cudaError_t alloc(size_t n) { return dmalloc(&p, std::max<size_t>(n, 16)); }
    ~DevBuf() {
        if (p) dfree(p);
    }
};

template <int DT>
cudaError_t run_adjoint(lbm_ctx* c, int T, int K, int plane_x, double* loss, double* dL_dg, int dg_on_device,
                        double* dL_dtau, bool* started) {
    using TT = typename Store<DT>::T;
    using R = Arith<DT>;
    cudaError_t e;
    const size_t copy = (size_t)c->n_sgroups * Q * GROUP_LANES * sizeof(TT);
    const int64_t n_slots = c->n_tiles * SLOTS;
    const bool grads = dL_dg || dL_dtau;
    const int n_ck = (T + K - 1) / K;
    const int seg_len = std::min(K, T);
    const size_t mu_bytes = (size_t)c->n_sgroups * Q * GROUP_LANES * sizeof(R);
    const int adj_blocks = (int)std::max<int64_t>(1, (c->n_own_nonsolid + ADJ_THREADS - 1) / ADJ_THREADS);
    const int nbl = (int)std::max<int64_t>(1, std::min<int64_t>((n_slots + LOSS_THREADS - 1) / LOSS_THREADS, 152 * 4));
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    // every buffer is allocated before any work, so that a failed allocation leaves the
    // state as it was: checkpoints (n_ck copies), one segment of recomputed states,
    // two adjoint buffers, the per-node and per-block FP64 gradient accumulators
    DevBuf ck, seg, mu0, mu1, gbar, taup, lossp, sums, dense;
    if ((e = lossp.alloc(sizeof(double) * 2 * nbl)) != cudaSuccess) return e;
    if ((e = sums.alloc(sizeof(double) * 2)) != cudaSuccess) return e;
    if (grads) {
        if ((e = ck.alloc(copy * n_ck)) != cudaSuccess) return e;
        if ((e = seg.alloc(copy * seg_len)) != cudaSuccess) return e;
        if ((e = mu0.alloc(mu_bytes)) != cudaSuccess) return e;
        if ((e = mu1.alloc(mu_bytes)) != cudaSuccess) return e;
        if ((e = gbar.alloc(sizeof(double) * n_slots)) != cudaSuccess) return e;
        if ((e = taup.alloc(sizeof(double) * adj_blocks)) != cudaSuccess) return e;
        if (dL_dg && !dg_on_device && (e = dense.alloc(N * sizeof(double))) != cudaSuccess) return e;
    }
    *started = true;
    // forward with checkpoints s_0, s_K, s_2K, ...
    for (int t = 0; t < T; t++) {
        if (grads && t % K == 0) {
            e = cudaMemcpyAsync(static_cast<char*>(ck.p) + copy * (t / K), c->f[c->cur], copy, cudaMemcpyDeviceToDevice,
                                c->stream);
            if (e != cudaSuccess) return e;
        }
        if ((e = launch_step(c, c->f[c->cur], c->f[1 - c->cur])) != cudaSuccess) return e;
        c->cur ^= 1;
    }
    // loss on s_T
    const TT* sT = static_cast<const TT*>(c->f[c->cur]);
    k_loss_partials<DT><<<nbl, LOSS_THREADS, 0, c->stream>>>(sT, c->nword, c->non_empty, c->smask, c->tlane, c->gfield,
                                                             c->n_tiles, c->Tx,
                                                             plane_x, c->p, static_cast<double*>(lossp.p));
    k_sum_partials<<<1, 32, 0, c->stream>>>(static_cast<const double*>(lossp.p), nbl, 2, static_cast<double*>(sums.p));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double h_sums[2] = {0.0, 0.0};
    if ((e = cudaMemcpyAsync(h_sums, sums.p, sizeof(h_sums), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    *loss = h_sums[1] > 0 ? h_sums[0] / h_sums[1] : 0.0;
    if (!grads || h_sums[1] == 0) {
        if (dL_dtau) *dL_dtau = 0.0;
        if (dL_dg && h_sums[1] == 0) {
            if (dg_on_device) e = cudaMemsetAsync(dL_dg, 0, N * sizeof(double), c->stream);
            else std::fill(dL_dg, dL_dg + N, 0.0);
        }
        return e;
    }
    // reverse sweep
    if ((e = cudaMemsetAsync(taup.p, 0, sizeof(double) * adj_blocks, c->stream)) != cudaSuccess) return e;
    R* mu[2] = {static_cast<R*>(mu0.p), static_cast<R*>(mu1.p)};
    int mcur = 0;
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_slots + 255) / 256, 152 * 32));
    k_loss_seed<DT><<<gs, 256, 0, c->stream>>>(sT, c->nword, c->non_empty, c->smask, c->tlane, c->gfield, c->n_tiles,
                                               c->Tx, plane_x, c->p,
                                               static_cast<const double*>(sums.p), mu[mcur],
                                               static_cast<double*>(gbar.p));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bool direct = true;
    for (int sgi = n_ck - 1; sgi >= 0; sgi--) {
        const int t0 = sgi * K, t1 = std::min(T, t0 + K);
        char* sb = static_cast<char*>(seg.p);
        if ((e = cudaMemcpyAsync(sb, static_cast<char*>(ck.p) + copy * sgi, copy, cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess)
            return e;
        for (int j = 1; j < t1 - t0; j++)
            if ((e = launch_step(c, sb + copy * (j - 1), sb + copy * j)) != cudaSuccess) return e;
        for (int t = t1 - 1; t >= t0; t--) {
            k_adjoint<DT><<<adj_blocks, ADJ_THREADS, 0, c->stream>>>(
                reinterpret_cast<const TT*>(sb + copy * (t - t0)), mu[mcur], direct ? 1 : 0, mu[1 - mcur], c->nbr,
                c->smask, c->tlane, c->fword, c->fidx, c->gfield, c->n_own_nonsolid, c->p, static_cast<double*>(gbar.p),
                static_cast<double*>(taup.p));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            mcur ^= 1;
            direct = false;
        }
    }
    if (dL_dtau) {
        k_sum_partials<<<1, 32, 0, c->stream>>>(static_cast<const double*>(taup.p), adj_blocks, 1,
                                                static_cast<double*>(sums.p));
        if ((e = cudaMemcpyAsync(dL_dtau, sums.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return e;
    }
    if (dL_dg) {
        double* d = dg_on_device ? dL_dg : static_cast<double*>(dense.p);
        if ((e = cudaMemsetAsync(d, 0, N * sizeof(double), c->stream)) != cudaSuccess) return e;
        k_gbar_dense<<<gs, 256, 0, c->stream>>>(static_cast<const double*>(gbar.p), c->nword, c->non_empty, c->n_tiles,
                                                c->nx, c->ny, c->Tx, c->Ty, d);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (!dg_on_device) {
            if ((e = cudaMemcpyAsync(dL_dg, d, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
                return e;
        }
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(c->stream);
}

}  // namespace

cudaError_t launch_adjoint(lbm_ctx* c, int T, int K, int plane_x, double* loss, double* dL_dg, int dg_on_device,
                           double* dL_dtau, bool* started) {
    *started = false;
    switch (c->dtype) {
        case LBM_F64: return run_adjoint<LBM_F64>(c, T, K, plane_x, loss, dL_dg, dg_on_device, dL_dtau, started);
        case LBM_F32: return run_adjoint<LBM_F32>(c, T, K, plane_x, loss, dL_dg, dg_on_device, dL_dtau, started);
        default: return run_adjoint<LBM_F16S>(c, T, K, plane_x, loss, dL_dg, dg_on_device, dL_dtau, started);
    }
}

}  // namespace lbm
