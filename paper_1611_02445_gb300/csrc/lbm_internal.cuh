// lbm_internal.cuh -- definitions shared by the translation units of liblbm_gb300.
//
// Device data layout (all in HBM, allocated once per context):
//   tile_map [Tz*Ty*Tx]  int32   rank of a kept tile, or -1 (Sec. 3.1 tileMap)
//   non_empty[n_tiles]   uint32  linear tile index t = tx + Tx (ty + Ty tz) (nonEmptyTiles)
//   nbr      [n_tiles][28] int32 ranks of the 3x3x3 tile neighbourhood, index
//                               13 + dx + 3 dy + 9 dz, -1 for dropped or out-of-box tiles
//                               (the local tileMap copy of Sec. 3.4, precomputed once);
//                               entry 27 is padding so each record is 112 bytes
//   nword    [n_tiles][64] uint32 per node: bit i (1..18) set when the gather of
//                               direction i bounces back (source solid, dropped or
//                               outside the box); bits 20-21 the node type
//   smask    [n_tiles]   uint64  bit s set when node s of the tile is solid or padding
//   tflags   [n_tiles]   uint32  bit 0: the tile holds inlet or outlet nodes
//   ntype    [n_tiles][64] uint8 node types in slot order (the per-tile nodeType block)
//   f[2]     [n_sgroups][19][256] populations of the non-solid nodes only, grouped: the
//                               kept tiles are cut into storage groups of consecutive
//                               tiles with at most 256 non-solid nodes (the step's work
//                               groups, plus those of a slab's ghost planes), and a group
//                               holds one 256-value data block per direction. A node's
//                               padded lane is P = 256 * group + its lane in the group;
//                               the lanes of a tile are consecutive in slot order, so the
//                               node in slot s of tile k has P = tlane[k] + (non-solid
//                               slots of the tile below s), and f_i lives at
//                               (P / 256) * 19 * 256 + 256 i + P % 256 (data_index)
//   tlane    [n_tiles]   int32   padded lane of each tile's first non-solid node
//   nrec     [n_tiles][28] int64 the step's neighbour records: for the 3x3x3 tile
//                               neighbourhood (index 13 + dx + 3 dy + 9 dz) the index in a
//                               copy of the neighbour's first non-solid node in data block
//                               0; zero for dropped or out-of-box tiles, which no gather
//                               reads (their links bounce back); entry 27 is padding so
//                               each record is 224 bytes, 16-byte aligned
//   gfield   [n_tiles][64]       optional per-node x force (double for F64, else float)
//   groups   [n_groups] int4     work units of the step kernel: {first tile, tiles (<= 16
//                               for FP64 storage, <= 8 otherwise), first fluid node, fluid
//                               nodes (<= 256)}, consecutive tiles; work group g is
//                               storage group sg0 + g
//   fword    [n_fluid] uint32    the gather word of every non-solid node in group order,
//                               plus bit 19 set when the node lies on the moving lid face
//                               (lbm_set_lid), bits 22-25 its tile within the group and
//                               bits 26-31 its slot
//   fidx     [n_fluid] uint32    k * 64 + s of every non-solid node in the same order
//   frank    [n_fluid] uint4     per node and pulled direction i (1..18) the rank of the
//                               source slot among its tile's non-solid slots, 6 bits each,
//                               five directions per word (rank_of); 0 for a bounced link.
//                               f_i(x - c_i) then lives at nrec[tile][nb] + 256 i + rank
//   gfield_c [n_fluid]           the per-node force in the same order
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_collide_df.cuh"

namespace lbm {

constexpr int Q = 19;
constexpr int TILE = 4;
constexpr int SLOTS = 64;
constexpr int NBR = 27;
constexpr int NBR_STRIDE = 28;   // padded neighbour record: 112 bytes, 16-byte aligned
constexpr int WORD_LID_BIT = 19;      // compact words: the node lies on the moving-wall face
constexpr int WORD_TYPE_SHIFT = 20;
constexpr int WORD_LT_SHIFT = 22;      // compact words: tile within the group (4 bits)
constexpr int WORD_LT_MASK = 15;
constexpr int WORD_SLOT_SHIFT = 26;    // compact words: slot in the tile (6 bits)
constexpr int GROUP_MAX_TILES_F64 = 16;   // tiles per work group: FP64 storage
constexpr int GROUP_MAX_TILES_4B = 8;     // and the 4-byte-or-smaller formats
constexpr int GRAPH_STEPS = 16;
// kernel kinds: the fused step and the paper's two calibration kernels (Sec. 4.1)
constexpr int STEP_FULL = 0;        // gather, collide, store
constexpr int STEP_PROPAGATE = 1;   // gather with bounce-back and store ("propagation only")
constexpr int STEP_RW = 2;          // read and write each node's own values ("read/write only")
constexpr int GROUP_MAX_NODES = 256;       // work-group size of the 4-byte-or-smaller formats
constexpr int GROUP_MAX_NODES_F64 = 256;   // and of FP64 storage (see the step kernel's CTA shape)
constexpr int GROUP_LANES = 256;           // lanes of a storage group: the length of its data blocks
constexpr int FLAG_HAS_BC = 1;
// F16S storage scale: h is stored as half(h * 2^12), so |h| in [1.5e-8, 16] is normal.
constexpr float F16_SCALE = 4096.0f;
constexpr float F16_INV_SCALE = 1.0f / 4096.0f;

// D3Q19 velocities in the numbering documented in lbm.h, weights of Sec. 2.2.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 10 || i == 11 || i == 12) ? 1
         : (i == 3 || i == 8 || i == 9 || i == 13 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 7 || i == 8 || i == 15 || i == 16) ? 1
         : (i == 4 || i == 9 || i == 10 || i == 17 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 13 || i == 15 || i == 17) ? 1
         : (i == 6 || i == 12 || i == 14 || i == 16 || i == 18) ? -1 : 0;
}
// Opposite direction (c_inv(i) = -c_i): 1<->3, 2<->4, 5<->6, 7<->9, 8<->10, 11<->14,
// 12<->13, 15<->18, 16<->17; constexpr so that it folds after unrolling.
__host__ __device__ constexpr int inv(int i) {
    return i == 1 ? 3 : i == 3 ? 1 : i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 6 : i == 6 ? 5
         : i == 7 ? 9 : i == 9 ? 7 : i == 8 ? 10 : i == 10 ? 8 : i == 11 ? 14 : i == 14 ? 11
         : i == 12 ? 13 : i == 13 ? 12 : i == 15 ? 18 : i == 18 ? 15 : i == 16 ? 17
         : i == 17 ? 16 : 0;
}
__host__ __device__ constexpr double wgt(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Index of f_i of the node with padded lane P in a copy of the populations (the grouped
// layout above): data block i of storage group P / 256, position P % 256.
__host__ __device__ inline int64_t data_index(uint32_t P, int i) {
    return (int64_t)(P / GROUP_LANES) * (Q * GROUP_LANES) + i * GROUP_LANES + (P % GROUP_LANES);
}
// Rank of direction i's source slot (i = 1..18) in a node's rank words (frank).
__host__ __device__ inline uint32_t rank_of(const uint4& r, int i) {
    const int w = (i - 1) / 5, b = 6 * ((i - 1) % 5);
    const uint32_t v = w == 0 ? r.x : w == 1 ? r.y : w == 2 ? r.z : r.w;
    return (v >> b) & 63u;
}
// Padded lane of the non-solid slot s of a tile whose first non-solid node has padded
// lane tl and whose solid mask is sm: tl plus the non-solid slots below s.
__device__ __forceinline__ uint32_t node_lane(uint32_t tl, uint64_t sm, int s) {
    return tl + (uint32_t)__popcll(~sm & ((1ull << s) - 1ull));
}

// Storage traits: element type T in HBM and arithmetic type R.
template <int DT> struct Store;
template <> struct Store<LBM_F64> {
    using T = double;
    using R = double;
    static constexpr bool SHIFT = false;   // arithmetic on f itself
};
template <> struct Store<LBM_F32> {
    using T = float;
    using R = float;
    static constexpr bool SHIFT = true;    // arithmetic and storage on h = f - w
};
template <> struct Store<LBM_F16S> {
    using T = __half;
    using R = float;
    static constexpr bool SHIFT = true;    // arithmetic and storage on h = f - w
};

inline size_t dtype_size(int dt) { return dt == LBM_F64 ? 8 : dt == LBM_F32 ? 4 : 2; }

struct StepParams {
    double omega;   // 1/tau
    double beta;    // 1 - 1/(2 tau), Guo prefactor
    double g[3];
    double u_in[3];
    double rho_out;
    const void* gfield;
    DFConst dfc;   // constants of the double-float FP64 collision
    DFClosure dfb; // and of its inlet and outlet closures
    // FP32 copies for the 4-byte formats (an FP64 -> FP32 conversion runs on the FP64 pipe)
    float omega_f, beta_f, g_f[3], u_in_f[3], rho_out_f, rho_out_m1_f;
    // collision model (lbm_set_model): equilibrium (LBM_EQ_*) and collision (LBM_COLL_*);
    // for MRT, moment k relaxes as m*_k = m^eq_k + (1 - s_k)(m_k - m^eq_k) + (1 - s_k/2) mG_k,
    // kept as mrt_a[k] = (1 - s_k) / |M_k|^2 and mrt_b[k] = (1 - s_k/2) / |M_k|^2
    int eq, coll;
    double mrt_a[Q], mrt_b[Q];
    float mrt_a_f[Q], mrt_b_f[Q];
    // moving wall (lbm_set_lid): 6 w_i (c_i . u_lid) for the directions whose links cross
    // the lid face from a node on it, 0 for the others
    double lid_c[Q];
    float lid_c_f[Q];
    // boundary scheme of the inlet/outlet nodes (lbm_set_bc): LBM_BC_EQUILIBRIUM or
    // LBM_BC_ZOU_HE with the box faces of the inlet and the outlet nodes
    int bc;
    int zh_face[2];
    // storage group of work group 0 (a slab's lower ghost plane has groups before it)
    int64_t sg0;
    // always 0: the step kernel ANDs it with the values a thread has read from its staging
    // column and adds the result to the shared address the next gathers copy into, which
    // orders them after the reads (the compiler cannot fold it away)
    uint32_t zero;
    // extents the checked build (LBM_CHECKED) tests every index against (kept tiles,
    // non-solid nodes of the work groups, padded lanes of a copy), and its error word
    // (NULL in the normal build): the first failed check stores (code << 56) | value
    int64_t n_tiles, n_lanes, n_padded;
    unsigned long long* check;
};

// Codes of the checked build's error word.
enum : unsigned {
    CHECK_HEADER = 1,      // a work-group header outside the context's arrays
    CHECK_OWN_TILE = 2,    // a node word whose tile is not in its group
    CHECK_NEIGHBOUR = 3    // a pulled direction whose source lane lies outside the copy
};

// A parameter in the arithmetic type R: the FP64 value or its FP32 copy.
template <typename R> __host__ __device__ inline R par(double d, float f);
template <> __host__ __device__ inline double par<double>(double d, float) { return d; }
template <> __host__ __device__ inline float par<float>(double, float f) { return f; }

}  // namespace lbm

struct lbm_ctx {
    int nx = 0, ny = 0, nz = 0, Tx = 0, Ty = 0, Tz = 0;
    unsigned periodic = 0;
    int dtype = LBM_F64;        // storage format (LBM_F64, LBM_F32, LBM_F16S)
    bool native64 = false;      // LBM_F64_NATIVE: FP64 arithmetic throughout
    bool sr = false;            // LBM_F16S_SR: stochastic rounding of the step's stores
    bool gen = false;           // a collision model other than quasi-compressible LBGK
    double mrt_user[5] = {1.19, 1.4, 1.2, 1.4, 1.98};   // s_e, s_eps, s_q, s_pi, s_m
    int lid_face = -1;          // moving box face (lbm_set_lid), -1 for none
    int bc = 0;                 // inlet/outlet scheme (lbm_set_bc)
    uint32_t* seed = nullptr;   // step counters of the rounding hash, one per copy
    unsigned long long* check = nullptr;   // error word of the checked build (LBM_CHECKED), else NULL
    int64_t n_tiles = 0, n_nonsolid = 0;
    // Tiles the step updates, reduces and exports: ranks [own_k0, own_k1). All of them in
    // a whole-domain context; a slab context (lbm_create_slab) also holds one ghost tile
    // plane below and/or above its own planes (ranks [0, own_k0) and [own_k1, n_tiles)),
    // which only receive the neighbours' boundary data.
    int64_t own_k0 = 0, own_k1 = 0;
    int ghost_lo = 0, ghost_hi = 0;     // ghost tile planes at the bottom / top of the box
    int64_t bnd_lo = 0, bnd_hi = 0;     // kept tiles in the lowest / highest own tile plane
    int z_plane0 = 0;                   // global tile plane of the box's first plane (slab)
    int64_t n_own_nonsolid = 0;         // non-solid nodes of the own tiles
    cudaStream_t stream = nullptr;
    int32_t* tile_map = nullptr;
    uint32_t* non_empty = nullptr;
    int32_t* nbr = nullptr;
    uint64_t* smask = nullptr;
    uint32_t* tflags = nullptr;
    uint8_t* ntype = nullptr;
    uint32_t* nword = nullptr;
    int4* groups = nullptr;
    uint32_t* fword = nullptr;
    uint32_t* fidx = nullptr;
    int32_t* tlane = nullptr;
    int64_t* nrec = nullptr;
    uint4* frank = nullptr;
    int64_t n_sgroups = 0;      // storage groups of a copy (work groups and ghost-plane groups)
    void* gfield_c = nullptr;
    int64_t n_groups = 0;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void* gfield = nullptr;
    bool params_set = false;
    bool state_set = false;
    lbm::StepParams p{};
    double tau = 0.0;
    // reduction scratch
    double* partials = nullptr;
    double* d_out = nullptr;
    int n_partials = 0;
    uint64_t geometry_hash = 0;
    // CUDA graphs of GRAPH_STEPS consecutive steps, one per starting copy (0 or 1)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool use_graphs = true;
    lbm_status sticky = LBM_OK;
    std::string err;
};

namespace lbm {
// Every device buffer of the library is allocated and released through these two
// (lbm_capi.cu): they count live buffers, and the host-side test hook of lbm_testing.h
// can make the k-th allocation fail as cudaMalloc does when memory runs out.
cudaError_t dmalloc(void** p, size_t bytes);
void dfree(void* p);

// Launchers (defined in lbm_tiles.cu / lbm_step.cu); all queue work on ctx->stream and
// return cudaGetLastError() of the launch.
cudaError_t launch_tile_flags(const uint8_t* nt, int nx, int ny, int nz, int Tx, int Ty, int Tz,
                              uint8_t* flag, int* bad, cudaStream_t st);
cudaError_t launch_scan_flags(const uint8_t* flag, int64_t n, int32_t* tile_map, uint32_t* non_empty,
                              int64_t* d_count, int64_t* block_sums, int64_t nblocks, cudaStream_t st);
int64_t scan_block_count(int64_t n);
cudaError_t launch_tile_meta(lbm_ctx* c, const uint8_t* nt);
cudaError_t launch_node_words(lbm_ctx* c);
cudaError_t launch_lane_lists(lbm_ctx* c, const int64_t* lane0, const uint8_t* lt);
cudaError_t launch_node_records(lbm_ctx* c);
cudaError_t launch_init(lbm_ctx* c, double rho0, const double u0[3]);
cudaError_t launch_step(lbm_ctx* c, const void* A, void* B);
cudaError_t launch_step_kind(lbm_ctx* c, int kind, const void* A, void* B);
cudaError_t prepare_step(lbm_ctx* c);
cudaError_t launch_reduce(lbm_ctx* c, double* d_out);
cudaError_t launch_macroscopic(lbm_ctx* c, void* rho, void* u, int out_f64);
cudaError_t launch_get_box(lbm_ctx* c, int x0, int y0, int z0, int bx, int by, int bz, double* d_out);
cudaError_t launch_halo(lbm_ctx* c, int side, int pack, void* buf);
cudaError_t launch_set_dense(lbm_ctx* c, const double* d_dense);
cudaError_t launch_gfield(lbm_ctx* c, const double* d_dense);
cudaError_t launch_gfield_compact(lbm_ctx* c);
cudaError_t launch_mark_lid(lbm_ctx* c, int face);
cudaError_t launch_adjoint(lbm_ctx* c, int T, int K, int plane_x, double* loss, double* dL_dg, int dg_on_device,
                           double* dL_dtau, bool* started);
}  // namespace lbm
