// lbm_tiles.cu -- tile-map builder (Algorithm 1 on the GPU), per-tile metadata,
// equilibrium initialisation, FP64 invariant reduction, macroscopic export and the
// dense <-> tile-major conversions of liblbm_gb300.
#include <algorithm>

#include "lbm_internal.cuh"
#include "lbm_df.cuh"
#include "lbm_store.cuh"

namespace lbm {

// ----------------------------------------------------------------------------------
// Algorithm 1 (Sec. 3.1) as flag -> exclusive scan -> scatter. The scan runs over the
// linear tile index t = tx + Tx (ty + Ty tz), which is the loop order of Algorithm 1,
// so ranks equal the paper's discovery order.

// flag[t] = 1 when some node of tile t is not solid; padding nodes count as solid.
__global__ void k_tile_flags(const uint8_t* __restrict__ nt, int nx, int ny, int nz, int Tx, int Ty,
                             int Tz, uint8_t* __restrict__ flag, int* __restrict__ bad) {
    const int64_t nT = (int64_t)Tx * Ty * Tz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nT;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int tx = (int)(t % Tx);
        const int64_t r = t / Tx;
        const int ty = (int)(r % Ty);
        const int tz = (int)(r / Ty);
        int any = 0, badv = 0;
        for (int dz = 0; dz < TILE; dz++) {
            const int z = TILE * tz + dz;
            if (z >= nz) break;
            for (int dy = 0; dy < TILE; dy++) {
                const int y = TILE * ty + dy;
                if (y >= ny) break;
                const uint8_t* row = nt + ((int64_t)z * ny + y) * nx;
                for (int dx = 0; dx < TILE; dx++) {
                    const int x = TILE * tx + dx;
                    if (x >= nx) break;
                    const uint8_t v = row[x];
                    any |= (v != LBM_SOLID);
                    badv |= (v > LBM_OUTLET);
                }
            }
        }
        flag[t] = (uint8_t)any;
        if (badv) atomicOr(bad, 1);
    }
}

constexpr int SCAN_BLOCK = 1024;

// Exclusive prefix sum of v over the 1024 threads of a block; *total gets the sum.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;   // inclusive over warps
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    *total = warp_sums[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(const uint8_t* __restrict__ flag, int64_t n,
                                                          int64_t* __restrict__ block_sums) {
    const int64_t t = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
    const int64_t v = t < n ? flag[t] : 0;
    int64_t total;
    block_exclusive_scan(v, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the block sums in chunks of 1024 with a running carry.
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_top(int64_t* __restrict__ block_sums, int64_t nb,
                                                         int64_t* __restrict__ d_count) {
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_BLOCK) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? block_sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, &total);
        if (i < nb) block_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *d_count = carry;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_scatter(const uint8_t* __restrict__ flag, int64_t n,
                                                             const int64_t* __restrict__ block_off,
                                                             int32_t* __restrict__ tile_map,
                                                             uint32_t* __restrict__ non_empty) {
    const int64_t t = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
    const int64_t v = t < n ? flag[t] : 0;
    int64_t total;
    const int64_t rank = block_off[blockIdx.x] + block_exclusive_scan(v, &total);
    if (t < n) {
        tile_map[t] = v ? (int32_t)rank : -1;
        if (v) non_empty[rank] = (uint32_t)t;
    }
}

int64_t scan_block_count(int64_t n) { return (n + SCAN_BLOCK - 1) / SCAN_BLOCK; }

cudaError_t launch_tile_flags(const uint8_t* nt, int nx, int ny, int nz, int Tx, int Ty, int Tz,
                              uint8_t* flag, int* bad, cudaStream_t st) {
    const int64_t nT = (int64_t)Tx * Ty * Tz;
    const int64_t blocks = std::min<int64_t>((nT + 255) / 256, 152 * 64);
    k_tile_flags<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(nt, nx, ny, nz, Tx, Ty, Tz, flag, bad);
    return cudaGetLastError();
}

cudaError_t launch_scan_flags(const uint8_t* flag, int64_t n, int32_t* tile_map, uint32_t* non_empty,
                              int64_t* d_count, int64_t* block_sums, int64_t nblocks, cudaStream_t st) {
    k_scan_sums<<<(unsigned)nblocks, SCAN_BLOCK, 0, st>>>(flag, n, block_sums);
    k_scan_top<<<1, SCAN_BLOCK, 0, st>>>(block_sums, nblocks, d_count);
    k_scan_scatter<<<(unsigned)nblocks, SCAN_BLOCK, 0, st>>>(flag, n, block_sums, tile_map, non_empty);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Per-tile metadata: node types in slot order, the solid mask, the boundary flag and
// the 3x3x3 neighbourhood of tile ranks (the local tileMap copy of Sec. 3.4), wrapped on
// periodic axes. One 64-thread block per kept tile, thread s = slot s.
__global__ void __launch_bounds__(64) k_tile_meta(const uint8_t* __restrict__ nt, int nx, int ny, int nz,
                                                  int Tx, int Ty, int Tz, unsigned periodic,
                                                  const int32_t* __restrict__ tile_map,
                                                  const uint32_t* __restrict__ non_empty, int64_t n_tiles,
                                                  int32_t* __restrict__ nbr, uint64_t* __restrict__ smask,
                                                  uint32_t* __restrict__ tflags, uint8_t* __restrict__ ntype,
                                                  unsigned long long* __restrict__ n_nonsolid) {
    __shared__ uint32_t s_solid[2], s_bc[2];
    const int s = threadIdx.x, lane = s & 31, warp = s >> 5;
    for (int64_t k = blockIdx.x; k < n_tiles; k += gridDim.x) {
        const uint32_t t = non_empty[k];
        const int tx = (int)(t % (uint32_t)Tx);
        const int ty = (int)((t / (uint32_t)Tx) % (uint32_t)Ty);
        const int tz = (int)(t / ((uint32_t)Tx * (uint32_t)Ty));
        const int x = TILE * tx + (s & 3), y = TILE * ty + ((s >> 2) & 3), z = TILE * tz + (s >> 4);
        uint8_t v = LBM_SOLID;
        if (x < nx && y < ny && z < nz) v = nt[x + (int64_t)nx * (y + (int64_t)ny * z)];
        ntype[k * SLOTS + s] = v;
        const uint32_t solid_bits = __ballot_sync(0xffffffffu, v == LBM_SOLID);
        const uint32_t bc_bits = __ballot_sync(0xffffffffu, v == LBM_INLET || v == LBM_OUTLET);
        if (lane == 0) {
            s_solid[warp] = solid_bits;
            s_bc[warp] = bc_bits;
            atomicAdd(n_nonsolid, (unsigned long long)(32 - __popc(solid_bits)));
        }
        if (s < NBR) {
            const int d[3] = {s % 3 - 1, (s / 3) % 3 - 1, s / 9 - 1};
            int c[3] = {tx + d[0], ty + d[1], tz + d[2]};
            const int T[3] = {Tx, Ty, Tz};
            bool inside = true;
            for (int a = 0; a < 3; a++) {
                if (c[a] < 0 || c[a] >= T[a]) {
                    if (periodic & (1u << a)) c[a] = (c[a] + T[a]) % T[a];
                    else inside = false;
                }
            }
            nbr[k * NBR_STRIDE + s] = inside ? tile_map[c[0] + (int64_t)Tx * (c[1] + (int64_t)Ty * c[2])] : -1;
        } else if (s == NBR) {
            nbr[k * NBR_STRIDE + s] = -1;
        }
        __syncthreads();
        if (s == 0) {
            smask[k] = (uint64_t)s_solid[0] | ((uint64_t)s_solid[1] << 32);
            tflags[k] = (s_bc[0] | s_bc[1]) ? FLAG_HAS_BC : 0;
        }
        __syncthreads();
    }
}

cudaError_t launch_tile_meta(lbm_ctx* c, const uint8_t* nt) {
    unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(c->d_out);
    cudaError_t e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>(c->n_tiles, 1 << 20);
    if (blocks > 0)
        k_tile_meta<<<(unsigned)blocks, 64, 0, c->stream>>>(nt, c->nx, c->ny, c->nz, c->Tx, c->Ty, c->Tz,
                                                            c->periodic, c->tile_map, c->non_empty,
                                                            c->n_tiles, c->nbr, c->smask, c->tflags,
                                                            c->ntype, d_cnt);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Per-node gather words: for every non-solid node, which of the 18 moving directions
// bounce back (their source x - c_i is solid, in a dropped tile or outside a
// non-periodic box), plus the node type. Built once; the step kernel then needs no
// neighbour masks.
__global__ void __launch_bounds__(64) k_node_words(const int32_t* __restrict__ nbr, const uint64_t* __restrict__ smask,
                                                   const uint8_t* __restrict__ ntype, int64_t n_tiles,
                                                   uint32_t* __restrict__ nword) {
    const int s = threadIdx.x;
    const int x = s & 3, y = (s >> 2) & 3, z = s >> 4;
    for (int64_t k = blockIdx.x; k < n_tiles; k += gridDim.x) {
        const uint32_t type = ntype[k * SLOTS + s];
        uint32_t w = 0;
        if (type != LBM_SOLID) {
            w = type << WORD_TYPE_SHIFT;
#pragma unroll
            for (int i = 1; i < Q; i++) {
                const int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);
                const int nb = 13 + (sx >> 2) + 3 * (sy >> 2) + 9 * (sz >> 2);
                const int ss = (sx & 3) | ((sy & 3) << 2) | ((sz & 3) << 4);
                const int32_t nk = nbr[k * NBR_STRIDE + nb];
                const bool bounce = nk < 0 || ((smask[nk] >> ss) & 1);
                if (bounce) w |= 1u << i;
            }
        }
        nword[k * SLOTS + s] = w;
    }
}

cudaError_t launch_node_words(lbm_ctx* c) {
    const int64_t blocks = std::min<int64_t>(c->n_tiles, 1 << 20);
    if (blocks > 0) k_node_words<<<(unsigned)blocks, 64, 0, c->stream>>>(c->nbr, c->smask, c->ntype, c->n_tiles, c->nword);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Equilibrium initial state f = f^eq(rho0, u0) (Eq. 3) of every non-solid node, in both
// copies.
template <int DT>
__global__ void k_init(typename Store<DT>::T* __restrict__ f0, typename Store<DT>::T* __restrict__ f1,
                       const uint64_t* __restrict__ smask, const int32_t* __restrict__ tlane, int64_t n_tiles,
                       double rho0, double ux, double uy, double uz, int eq) {
    using T = typename Store<DT>::T;
    const int64_t n = n_tiles * SLOTS;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const uint64_t sm = smask[k];
        if ((sm >> s) & 1) continue;   // solid slots have no storage
        const uint32_t P = node_lane((uint32_t)tlane[k], sm, s);
        const double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
            // Eq. 3, or Eq. 4 for the incompressible model
            const double fe = eq == LBM_EQ_INCOMPR ? wgt(i) * (rho0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)
                                                   : wgt(i) * rho0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            const T v = from_f64<DT>(fe, i);
            f0[data_index(P, i)] = v;
            f1[data_index(P, i)] = v;
        }
    }
}

// The per-lane lists of the step's work groups (fword, fidx), from what the host decided
// per tile while forming the groups: the non-solid nodes of tile k take lanes lane0[k],
// lane0[k] + 1, ... in slot order, and lt[k] is the tile's index within its group. One CTA
// of 64 threads per tile, one thread per slot; a slot's rank is the popcount of the
// tile's non-solid mask below it.
__global__ void k_lane_lists(const uint32_t* __restrict__ nword, const uint64_t* __restrict__ smask,
                             const int32_t* __restrict__ nbr, const int64_t* __restrict__ lane0,
                             const uint8_t* __restrict__ lt, int64_t k0, int64_t k1, uint32_t* __restrict__ fword,
                             uint32_t* __restrict__ fidx, uint4* __restrict__ frank) {
    const int s = threadIdx.x;
    const int x = s & 3, y = (s >> 2) & 3, z = s >> 4;
    const uint64_t below = (1ull << s) - 1ull;   // s < 64
    for (int64_t k = k0 + blockIdx.x; k < k1; k += gridDim.x) {
        const uint64_t sm = smask[k];
        const uint32_t l = lt[k - k0];
        if (!((sm >> s) & 1ull)) {
            const int64_t idx = lane0[k - k0] + __popcll(~sm & below);
            const uint32_t w = nword[k * SLOTS + s];
            fword[idx] = w | (l << WORD_LT_SHIFT) | ((uint32_t)s << WORD_SLOT_SHIFT);
            fidx[idx] = (uint32_t)(k * SLOTS + s);
            uint32_t r[4] = {0u, 0u, 0u, 0u};
            for (int i = 1; i < Q; i++) {
                if ((w >> i) & 1u) continue;   // bounced: no source in another slot
                const int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);
                const int nb = 13 + (sx >> 2) + 3 * (sy >> 2) + 9 * (sz >> 2);
                const int ss = (sx & 3) | ((sy & 3) << 2) | ((sz & 3) << 4);
                const int32_t nk = nbr[k * NBR_STRIDE + nb];   // >= 0: the link does not bounce
                const uint32_t rank = (uint32_t)__popcll(~smask[nk] & ((1ull << ss) - 1ull));
                r[(i - 1) / 5] |= rank << (6 * ((i - 1) % 5));
            }
            frank[idx] = make_uint4(r[0], r[1], r[2], r[3]);
        }
    }
}

cudaError_t launch_lane_lists(lbm_ctx* c, const int64_t* lane0, const uint8_t* lt) {
    const int64_t n = c->own_k1 - c->own_k0;
    if (n <= 0) return cudaSuccess;
    k_lane_lists<<<(unsigned)std::min<int64_t>(n, 1 << 20), SLOTS, 0, c->stream>>>(
        c->nword, c->smask, c->nbr, lane0, lt, c->own_k0, c->own_k1, c->fword, c->fidx, c->frank);
    return cudaGetLastError();
}

// The step's neighbour records: for each kept tile and each of its 27 neighbourhood
// entries, the index of the neighbour's first non-solid node in data block 0 of a copy
// (zero for a dropped or out-of-box neighbour, and in the padding entry). One thread per
// record.
__global__ void k_node_records(const int32_t* __restrict__ nbr, const int32_t* __restrict__ tlane, int64_t n_tiles,
                               int64_t* __restrict__ nrec) {
    const int64_t n = n_tiles * NBR_STRIDE;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx % NBR_STRIDE);
        const int32_t r = e < NBR ? nbr[idx] : -1;
        nrec[idx] = r >= 0 && r < n_tiles ? data_index((uint32_t)tlane[r], 0) : 0;
    }
}

static unsigned grid_for(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32));
}

cudaError_t launch_node_records(lbm_ctx* c) {
    if (c->n_tiles <= 0) return cudaSuccess;
    k_node_records<<<grid_for(c->n_tiles * NBR_STRIDE, 256), 256, 0, c->stream>>>(c->nbr, c->tlane, c->n_tiles,
                                                                                 c->nrec);
    return cudaGetLastError();
}

cudaError_t launch_init(lbm_ctx* c, double rho0, const double u0[3]) {
    const unsigned g = grid_for(c->n_tiles * SLOTS, 256);
    switch (c->dtype) {
        case LBM_F64:
            k_init<LBM_F64><<<g, 256, 0, c->stream>>>((double*)c->f[0], (double*)c->f[1], c->smask, c->tlane,
                                                      c->n_tiles, rho0, u0[0], u0[1], u0[2], c->p.eq);
            break;
        case LBM_F32:
            k_init<LBM_F32><<<g, 256, 0, c->stream>>>((float*)c->f[0], (float*)c->f[1], c->smask, c->tlane,
                                                      c->n_tiles, rho0, u0[0], u0[1], u0[2], c->p.eq);
            break;
        default:
            k_init<LBM_F16S><<<g, 256, 0, c->stream>>>((__half*)c->f[0], (__half*)c->f[1], c->smask, c->tlane,
                                                       c->n_tiles, rho0, u0[0], u0[1], u0[2], c->p.eq);
    }
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// FP64 mass and momentum: per-thread FP64 partials -> warp shuffle tree -> one partial
// per block -> a fixed-order single-block pass. No atomics, so the result depends only
// on the launch shape, which is fixed per context.
constexpr int RED_THREADS = 256;

// Moments of one node as doubles: rho (or rho - 1 for the shifted formats, whose f is w + h
// with sum w = 1) and j. FP64 storage: exact sums of the values in 64-bit fixed point
// (2^-58), rounded once. FP32 / FP16 storage: the h values are FP32 numbers, summed with
// Knuth's TwoSum so that each moment is the rounded pair hi + lo (relative error ~2^-48).
// Either way each moment costs one or two FP64 operations, not 19: FP64 runs on 2 lanes
// per SM.
__device__ __forceinline__ float red_add(float a, float b, float& err) {
    const float sum = __fadd_rn(a, b);
    const float bb = __fsub_rn(sum, a);
    err = __fadd_rn(err, __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb)));
    return sum;
}

template <int DT>
__device__ __forceinline__ void node_moments(const typename Store<DT>::T* __restrict__ f, uint32_t P, double m[4]) {
    if constexpr (DT == LBM_F64) {
        // exact fixed-point sums; the conversion maps NaN and Inf to finite integers, so
        // a non-finite population is tested for on its exponent bits and makes every
        // moment of the node NaN (what the mass watchdog of lbm_reduce looks for)
        int64_t r = 0, jx = 0, jy = 0, jz = 0;
        uint64_t nonfinite = 0;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const double v = f[data_index(P, i)];
            const uint64_t b = (uint64_t)__double_as_longlong(v);
            nonfinite |= (~b & 0x7ff0000000000000ull) == 0 ? 1ull : 0ull;
            const int64_t q = fix_from_double(v);
            r += q;
            if (cx(i)) jx += cx(i) > 0 ? q : -q;
            if (cy(i)) jy += cy(i) > 0 ? q : -q;
            if (cz(i)) jz += cz(i) > 0 ? q : -q;
        }
        const double sc = 1.0 / (double)(1ull << FIX_SHIFT);
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        m[0] = nonfinite ? nan : __ll2double_rn(r) * sc;
        m[1] = nonfinite ? nan : __ll2double_rn(jx) * sc;
        m[2] = nonfinite ? nan : __ll2double_rn(jy) * sc;
        m[3] = nonfinite ? nan : __ll2double_rn(jz) * sc;
    } else {
        float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, er = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const float h = to_arith<DT>(f[data_index(P, i)], i);
            r = red_add(r, h, er);
            if (cx(i)) jx = red_add(jx, cx(i) > 0 ? h : -h, ex);
            if (cy(i)) jy = red_add(jy, cy(i) > 0 ? h : -h, ey);
            if (cz(i)) jz = red_add(jz, cz(i) > 0 ? h : -h, ez);
        }
        m[0] = 1.0 + ((double)r + (double)er);
        m[1] = (double)jx + (double)ex;
        m[2] = (double)jy + (double)ey;
        m[3] = (double)jz + (double)ez;
    }
}

template <int DT>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(const typename Store<DT>::T* __restrict__ f,
                                                        const uint64_t* __restrict__ smask,
                                                        const int32_t* __restrict__ tlane,
                                                        const void* __restrict__ gfield, int64_t n_tiles,
                                                        StepParams p, double* __restrict__ partials) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t n = n_tiles * SLOTS;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const uint64_t sm = smask[k];
        if ((sm >> s) & 1) continue;
        double m[4];
        node_moments<DT>(f, node_lane((uint32_t)tlane[k], sm, s), m);
        const double Fx = gfield ? gfield_at<DT>(gfield, idx) : p.g[0];
        acc[0] += m[0];
        acc[1] += m[1] - 0.5 * Fx;
        acc[2] += m[2] - 0.5 * p.g[1];
        acc[3] += m[3] - 0.5 * p.g[2];
    }
    __shared__ double sh[RED_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        double v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < RED_THREADS / 32; w++) v += sh[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double* __restrict__ partials, int nb,
                                                              double* __restrict__ out) {
    __shared__ double sh[RED_THREADS][4];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += RED_THREADS)
        for (int c = 0; c < 4; c++) acc[c] += partials[b * 4 + c];
    for (int c = 0; c < 4; c++) sh[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 4; c++) sh[threadIdx.x][c] += sh[threadIdx.x + h][c];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = sh[0][threadIdx.x];
}

int reduce_blocks(int64_t n_tiles) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n_tiles * SLOTS + RED_THREADS - 1) / RED_THREADS, 152 * 4));
}

// The own tiles of a context (all of them, or a slab context's without its ghost planes)
// as pointers to their first tile: populations, masks, tile indices and per-slot force.
struct OwnTiles {
    const void* f;
    const uint64_t* smask;
    const int32_t* tlane;
    const uint32_t* non_empty;
    const void* gfield;
    int64_t n;
};
static OwnTiles own_tiles(const lbm_ctx* c) {
    const int64_t k0 = c->own_k0;
    const size_t gsize = c->dtype == LBM_F64 ? 8 : 4;
    return {c->f[c->cur], c->smask + k0, c->tlane + k0, c->non_empty + k0, c->gfield ? static_cast<const char*>(c->gfield) + (size_t)k0 * SLOTS * gsize : nullptr,
            c->own_k1 - k0};
}

cudaError_t launch_reduce(lbm_ctx* c, double* d_out) {
    const int nb = c->n_partials;
    const OwnTiles o = own_tiles(c);
    switch (c->dtype) {
        case LBM_F64:
            k_reduce<LBM_F64><<<nb, RED_THREADS, 0, c->stream>>>((const double*)o.f, o.smask, o.tlane, o.gfield, o.n, c->p,
                                                                 c->partials);
            break;
        case LBM_F32:
            k_reduce<LBM_F32><<<nb, RED_THREADS, 0, c->stream>>>((const float*)o.f, o.smask, o.tlane, o.gfield, o.n, c->p,
                                                                 c->partials);
            break;
        default:
            k_reduce<LBM_F16S><<<nb, RED_THREADS, 0, c->stream>>>((const __half*)o.f, o.smask, o.tlane, o.gfield, o.n, c->p,
                                                                  c->partials);
    }
    k_reduce_final<<<1, RED_THREADS, 0, c->stream>>>(c->partials, nb, d_out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Macroscopic export from the stored post-collision populations: rho = sum f*,
// u = (sum c f* - F/2)/rho (Eq. 5; Eq. 6 without the division for the incompressible
// model), into dense arrays (already zeroed by the caller).
template <int DT, typename O>
__global__ void k_macro(const typename Store<DT>::T* __restrict__ f, const uint64_t* __restrict__ smask,
                        const int32_t* __restrict__ tlane, const uint32_t* __restrict__ non_empty,
                        const void* __restrict__ gfield,
                        int64_t n_tiles, int nx, int ny, int nz, int Tx, int Ty, StepParams p,
                        O* __restrict__ rho, O* __restrict__ u) {
    const int64_t n = n_tiles * SLOTS;
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const uint64_t sm = smask[k];
        if ((sm >> s) & 1) continue;
        const uint32_t t = non_empty[k];
        const int x = TILE * (int)(t % (uint32_t)Tx) + (s & 3);
        const int y = TILE * (int)((t / (uint32_t)Tx) % (uint32_t)Ty) + ((s >> 2) & 3);
        const int z = TILE * (int)(t / ((uint32_t)Tx * (uint32_t)Ty)) + (s >> 4);
        const int64_t node = x + (int64_t)nx * (y + (int64_t)ny * z);
        double m[4];
        node_moments<DT>(f, node_lane((uint32_t)tlane[k], sm, s), m);
        const double r = m[0], jx = m[1], jy = m[2], jz = m[3];
        const double Fx = gfield ? gfield_at<DT>(gfield, idx) : p.g[0];
        rho[node] = (O)r;
        if (p.eq == LBM_EQ_INCOMPR) {
            // Eq. 6: no division by the density
            u[node] = (O)(jx - 0.5 * Fx);
            u[N + node] = (O)(jy - 0.5 * p.g[1]);
            u[2 * N + node] = (O)(jz - 0.5 * p.g[2]);
        } else {
            u[node] = (O)((jx - 0.5 * Fx) / r);
            u[N + node] = (O)((jy - 0.5 * p.g[1]) / r);
            u[2 * N + node] = (O)((jz - 0.5 * p.g[2]) / r);
        }
    }
}

template <typename O>
static void macro_dispatch(lbm_ctx* c, O* rho, O* u) {
    const OwnTiles o = own_tiles(c);
    const unsigned g = grid_for(o.n * SLOTS, 256);
#define LBM_MACRO(DT, TT)                                                                                 \
    k_macro<DT, O><<<g, 256, 0, c->stream>>>((const TT*)o.f, o.smask, o.tlane, o.non_empty, o.gfield, o.n, c->nx, c->ny, \
                                             c->nz, c->Tx, c->Ty, c->p, rho, u)
    if (c->dtype == LBM_F64) LBM_MACRO(LBM_F64, double);
    else if (c->dtype == LBM_F32) LBM_MACRO(LBM_F32, float);
    else LBM_MACRO(LBM_F16S, __half);
#undef LBM_MACRO
}

cudaError_t launch_macroscopic(lbm_ctx* c, void* rho, void* u, int out_f64) {
    if (c->own_k1 <= c->own_k0) return cudaSuccess;
    if (out_f64) macro_dispatch<double>(c, (double*)rho, (double*)u);
    else macro_dispatch<float>(c, (float*)rho, (float*)u);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Box export: out[i][bz][by][bx] in FP64; NaN for solid, dropped or outside nodes.
template <int DT>
__global__ void k_get_box(const typename Store<DT>::T* __restrict__ f, const int32_t* __restrict__ tile_map,
                          const uint64_t* __restrict__ smask, const int32_t* __restrict__ tlane, int nx, int ny, int nz, int Tx, int Ty,
                          unsigned periodic, int x0, int y0, int z0, int bx, int by, int bz,
                          double* __restrict__ out) {
    const int64_t B = (int64_t)bx * by * bz;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        int p[3] = {x0 + (int)(b % bx), y0 + (int)((b / bx) % by), z0 + (int)(b / ((int64_t)bx * by))};
        const int n[3] = {nx, ny, nz};
        bool inside = true;
        for (int a = 0; a < 3; a++) {
            if (p[a] < 0 || p[a] >= n[a]) {
                if (periodic & (1u << a)) p[a] = ((p[a] % n[a]) + n[a]) % n[a];
                else inside = false;
            }
        }
        int64_t k = -1;
        uint32_t P = 0;
        if (inside) {
            k = tile_map[p[0] / TILE + (int64_t)Tx * (p[1] / TILE + (int64_t)Ty * (p[2] / TILE))];
            const int s = (p[0] & 3) + 4 * (p[1] & 3) + 16 * (p[2] & 3);
            if (k >= 0 && ((smask[k] >> s) & 1)) k = -1;
            if (k >= 0) P = node_lane((uint32_t)tlane[k], smask[k], s);
        }
#pragma unroll
        for (int i = 0; i < Q; i++)
            out[i * B + b] = k >= 0 ? to_f64<DT>(f[data_index(P, i)], i) : __longlong_as_double(0x7ff8000000000000ll);
    }
}

cudaError_t launch_get_box(lbm_ctx* c, int x0, int y0, int z0, int bx, int by, int bz, double* d_out) {
    const unsigned g = grid_for((int64_t)bx * by * bz, 256);
    const void* A = c->f[c->cur];
#define LBM_BOX(DT, TT)                                                                                   \
    k_get_box<DT><<<g, 256, 0, c->stream>>>((const TT*)A, c->tile_map, c->smask, c->tlane, c->nx, c->ny, c->nz, c->Tx, \
                                            c->Ty, c->periodic, x0, y0, z0, bx, by, bz, d_out)
    if (c->dtype == LBM_F64) LBM_BOX(LBM_F64, double);
    else if (c->dtype == LBM_F32) LBM_BOX(LBM_F32, float);
    else LBM_BOX(LBM_F16S, __half);
#undef LBM_BOX
    return cudaGetLastError();
}

// Dense FP64 import of the non-solid nodes into both copies.
template <int DT>
__global__ void k_set_dense(typename Store<DT>::T* __restrict__ f0, typename Store<DT>::T* __restrict__ f1,
                            const double* __restrict__ dense, const uint64_t* __restrict__ smask,
                            const int32_t* __restrict__ tlane, const uint32_t* __restrict__ non_empty,
                            int64_t n_tiles, int nx, int ny, int nz, int Tx, int Ty) {
    using T = typename Store<DT>::T;
    const int64_t n = n_tiles * SLOTS;
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const uint64_t sm = smask[k];
        if ((sm >> s) & 1) continue;   // solid slots have no storage
        const uint32_t P = node_lane((uint32_t)tlane[k], sm, s);
        const uint32_t t = non_empty[k];
        const int x = TILE * (int)(t % (uint32_t)Tx) + (s & 3);
        const int y = TILE * (int)((t / (uint32_t)Tx) % (uint32_t)Ty) + ((s >> 2) & 3);
        const int z = TILE * (int)(t / ((uint32_t)Tx * (uint32_t)Ty)) + (s >> 4);
        const int64_t node = x + (int64_t)nx * (y + (int64_t)ny * z);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const T v = from_f64<DT>(dense[i * N + node], i);
            f0[data_index(P, i)] = v;
            f1[data_index(P, i)] = v;
        }
    }
}

cudaError_t launch_set_dense(lbm_ctx* c, const double* d_dense) {
    const unsigned g = grid_for(c->n_tiles * SLOTS, 256);
#define LBM_SET(DT, TT)                                                                                   \
    k_set_dense<DT><<<g, 256, 0, c->stream>>>((TT*)c->f[c->cur], (TT*)c->f[1 - c->cur], d_dense, c->smask, \
                                              c->tlane, c->non_empty, c->n_tiles, c->nx, c->ny, c->nz, c->Tx, c->Ty)
    if (c->dtype == LBM_F64) LBM_SET(LBM_F64, double);
    else if (c->dtype == LBM_F32) LBM_SET(LBM_F32, float);
    else LBM_SET(LBM_F16S, __half);
#undef LBM_SET
    return cudaGetLastError();
}

// Dense per-node x force -> tile-major copy in the arithmetic precision.
template <typename G>
__global__ void k_gfield(G* __restrict__ gt, const double* __restrict__ dense, const uint32_t* __restrict__ non_empty,
                         int64_t n_tiles, int nx, int ny, int nz, int Tx, int Ty) {
    const int64_t n = n_tiles * SLOTS;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const uint32_t t = non_empty[k];
        const int x = TILE * (int)(t % (uint32_t)Tx) + (s & 3);
        const int y = TILE * (int)((t / (uint32_t)Tx) % (uint32_t)Ty) + ((s >> 2) & 3);
        const int z = TILE * (int)(t / ((uint32_t)Tx * (uint32_t)Ty)) + (s >> 4);
        const bool in = x < nx && y < ny && z < nz;
        gt[idx] = in ? (G)dense[x + (int64_t)nx * (y + (int64_t)ny * z)] : (G)0;
    }
}

// Tile-major force -> the compact per-fluid-node copy read by the step kernel.
template <typename G>
__global__ void k_gfield_compact(G* __restrict__ gc, const G* __restrict__ gt, const uint32_t* __restrict__ fidx,
                                 int64_t n_fluid) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_fluid; n += (int64_t)gridDim.x * blockDim.x)
        gc[n] = gt[fidx[n]];
}

cudaError_t launch_gfield_compact(lbm_ctx* c) {
    const unsigned g = grid_for(c->n_own_nonsolid, 256);
    if (c->dtype == LBM_F64)
        k_gfield_compact<double><<<g, 256, 0, c->stream>>>((double*)c->gfield_c, (const double*)c->gfield, c->fidx,
                                                           c->n_own_nonsolid);
    else
        k_gfield_compact<float><<<g, 256, 0, c->stream>>>((float*)c->gfield_c, (const float*)c->gfield, c->fidx,
                                                          c->n_own_nonsolid);
    return cudaGetLastError();
}

// Mark (or clear, face < 0) the compact words of the nodes on a box face: x = 0 (face 0),
// x = nx - 1 (1), y = 0 (2), y = ny - 1 (3), z = 0 (4), z = nz - 1 (5).
__global__ void k_mark_lid(uint32_t* __restrict__ fword, const uint32_t* __restrict__ fidx,
                           const uint32_t* __restrict__ non_empty, int64_t n_nodes, int Tx, int Ty, int nx, int ny,
                           int nz, int face) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_nodes;
         n += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t gi = fidx[n];
        const uint32_t t = non_empty[gi >> 6];
        const int s = (int)(gi & 63u);
        const int p[3] = {TILE * (int)(t % (uint32_t)Tx) + (s & 3),
                          TILE * (int)((t / (uint32_t)Tx) % (uint32_t)Ty) + ((s >> 2) & 3),
                          TILE * (int)(t / ((uint32_t)Tx * (uint32_t)Ty)) + (s >> 4)};
        const int dims[3] = {nx, ny, nz};
        bool on = false;
        if (face >= 0) {
            const int a = face >> 1;
            on = (face & 1) ? p[a] == dims[a] - 1 : p[a] == 0;
        }
        const uint32_t w = fword[n] & ~(1u << WORD_LID_BIT);
        fword[n] = on ? (w | (1u << WORD_LID_BIT)) : w;
    }
}

cudaError_t launch_mark_lid(lbm_ctx* c, int face) {
    if (c->n_own_nonsolid == 0) return cudaSuccess;
    k_mark_lid<<<grid_for(c->n_own_nonsolid, 256), 256, 0, c->stream>>>(c->fword, c->fidx, c->non_empty,
                                                                       c->n_own_nonsolid,
                                                                   c->Tx, c->Ty, c->nx, c->ny, c->nz, face);
    return cudaGetLastError();
}

cudaError_t launch_gfield(lbm_ctx* c, const double* d_dense) {
    const unsigned g = grid_for(c->n_tiles * SLOTS, 256);
    if (c->dtype == LBM_F64)
        k_gfield<double><<<g, 256, 0, c->stream>>>((double*)c->gfield, d_dense, c->non_empty, c->n_tiles, c->nx,
                                                   c->ny, c->nz, c->Tx, c->Ty);
    else
        k_gfield<float><<<g, 256, 0, c->stream>>>((float*)c->gfield, d_dense, c->non_empty, c->n_tiles, c->nx,
                                                  c->ny, c->nz, c->Tx, c->Ty);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Halo of a slab context (lbm_create_slab): the populations that cross the cut between
// two slabs. A node of the lowest own plane pulls from the plane below through the five
// directions with c_z = +1, one of the highest own plane from the plane above through
// the five with c_z = -1. Pack copies the own boundary plane's values of the directions
// its neighbour reads (side 0: the lowest plane, for the slab below, c_z = -1; side 1:
// the highest, for the slab above, c_z = +1) from the current copy into buf, laid out
// [direction][tile][64] with NaN in the solid slots; unpack copies the non-solid slots of
// buf into the ghost plane on that side (side 0: c_z = +1, side 1: c_z = -1). Both slabs
// hold the plane's tiles in the same order with the same masks, so the layout agrees.
struct HaloDirs {
    int d[5];
};

template <int DT>
__global__ void k_halo(typename Store<DT>::T* __restrict__ f, const uint64_t* __restrict__ smask,
                       const int32_t* __restrict__ tlane, int64_t n_tiles, HaloDirs dirs, int pack,
                       typename Store<DT>::T* __restrict__ buf) {
    const int64_t n = n_tiles * SLOTS;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx >> 6;
        const int s = (int)(idx & 63);
        const uint64_t sm = smask[k];
        const bool solid = (sm >> s) & 1;
        const uint32_t P = solid ? 0u : node_lane((uint32_t)tlane[k], sm, s);
#pragma unroll
        for (int d = 0; d < 5; d++) {
            if (pack) buf[d * n + idx] = solid ? nan_value<DT>() : f[data_index(P, dirs.d[d])];
            else if (!solid) f[data_index(P, dirs.d[d])] = buf[d * n + idx];
        }
    }
}

cudaError_t launch_halo(lbm_ctx* c, int side, int pack, void* buf) {
    HaloDirs down = {{6, 12, 14, 16, 18}};   // c_z = -1
    HaloDirs up = {{5, 11, 13, 15, 17}};     // c_z = +1
    int64_t k0, n;
    HaloDirs dirs;
    if (pack) {
        k0 = side == 0 ? c->own_k0 : c->own_k1 - c->bnd_hi;
        n = side == 0 ? c->bnd_lo : c->bnd_hi;
        dirs = side == 0 ? down : up;
    } else {
        k0 = side == 0 ? 0 : c->own_k1;
        n = side == 0 ? c->own_k0 : c->n_tiles - c->own_k1;
        dirs = side == 0 ? up : down;
    }
    if (n == 0) return cudaSuccess;
    const unsigned g = grid_for(n * SLOTS, 256);
#define LBM_HALO(DT, TT)                                                                                     \
    k_halo<DT><<<g, 256, 0, c->stream>>>((TT*)c->f[c->cur], c->smask + k0, c->tlane + k0, n, dirs, pack, (TT*)buf)
    if (c->dtype == LBM_F64) LBM_HALO(LBM_F64, double);
    else if (c->dtype == LBM_F32) LBM_HALO(LBM_F32, float);
    else LBM_HALO(LBM_F16S, __half);
#undef LBM_HALO
    return cudaGetLastError();
}

}  // namespace lbm
