/*
 * lbm.h -- C ABI of the GB300 (sm_103a) sparse-tile D3Q19 lattice-Boltzmann library.
 *
 * The library implements the fused collide-and-stream time step of Tomczak & Szafran,
 * "A new GPU implementation for lattice-Boltzmann simulations on sparse geometries":
 * the geometry is covered by a uniform grid of 4x4x4 tiles, tiles holding only solid
 * nodes are dropped (Sec. 3.1, Algorithm 1), and one kernel launch performs gather
 * (pull) streaming, boundary handling, LBGK collision and the store of all 19
 * populations for every non-solid node (Sec. 3.4, Algorithm 2; Eq. 7).
 *
 * Conventions shared by every entry point
 *   - Status: every call returns an lbm_status; no C++ exception crosses the ABI.
 *     Errors after which the device state is undefined (LBM_ECUDA, LBM_ENOMEM,
 *     LBM_EINTERNAL) are sticky: later calls on the context return the same status
 *     until lbm_destroy. Argument and ordering errors (LBM_EINVAL, LBM_EUNSUPPORTED,
 *     LBM_ESTATE) change nothing. lbm_last_error() gives a message.
 *   - Dense arrays are indexed n = x + nx*(y + ny*z) (x fastest, the row order of
 *     Sec. 3.2). Population arrays are [19][nz][ny][nx]; velocity arrays [3][nz][ny][nx].
 *   - Direction numbering: 0 rest; 1 E(+x) 2 N(+y) 3 W(-x) 4 S(-y) 5 T(+z) 6 B(-z);
 *     7 NE 8 NW 9 SW 10 SE; 11 ET 12 EB 13 WT 14 WB; 15 NT 16 NB 17 ST 18 SB
 *     (e_3 = W = (-1,0,0) as in the paper's Fig. 1; the rest of Fig. 1 is not legible).
 *   - Node types (one byte per node, the paper's allNodeType of Sec. 3.1): 0 solid,
 *     1 fluid, 2 velocity inlet, 3 constant-pressure outlet (boundary kinds of Sec. 2.2).
 *   - Ownership: the context owns every device buffer it allocates (populations,
 *     tile structures, checkpoints). The caller owns every pointer it passes; the
 *     library reads or writes them only during the call (device pointers on the
 *     context's stream, host pointers synchronously).
 *   - Streams: all device work is queued on the stream given to lbm_create (or
 *     lbm_set_stream); calls that return host results synchronise that stream.
 *   - Thread safety: a context must not be used from two threads at once.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,        /* invalid argument (sizes, tau <= 1/2, NaN parameters, ...) */
    LBM_ENOMEM = 2,        /* device or host allocation failed; nothing leaked */
    LBM_ECUDA = 3,         /* a CUDA runtime call failed */
    LBM_EUNSUPPORTED = 4,  /* valid but not implemented (tile size other than 4, ...) */
    LBM_ESTATE = 5,        /* call out of order, or a state blob that does not match */
    LBM_ENONFINITE = 6,    /* the mass reduction found NaN or Inf in the state */
    LBM_ETIMEOUT = 7,      /* reserved: a bounded device-side wait gave up */
    LBM_EINTERNAL = 8      /* internal consistency check failed */
} lbm_status;

/* Storage of the populations and the arithmetic of the step.
 *   LBM_F64         FP64 storage. The moments are exact 64-bit fixed-point sums of the
 *                   stored doubles and the final (1 - 1/tau) f + Y update runs in FP64;
 *                   Y = f^eq/tau + S runs in double-float (pairs of FP32, about 46-48
 *                   bits), because GB300's FP64 pipe has 2 lanes per SM. The equilibrium
 *                   inlet/outlet closures and the incompressible LBGK (lbm_set_model) use
 *                   the same arithmetic; MRT and the Zou-He completion run in FP64.
 *                   Agrees with FP64 arithmetic to ~1e-14 relative per step.
 *   LBM_F64_NATIVE  FP64 storage, every operation of the step in FP64.
 *   LBM_F32         stores h_i = f_i - w_i as FP32 (the equilibrium-weight shift),
 *                   FP32 arithmetic on h.
 *   LBM_F16S        stores h_i = (f_i - w_i) * 2^12 as IEEE binary16 (round to nearest
 *                   even), FP32 arithmetic on h. The step's stores carry each node's
 *                   rounding residue of mass into direction 0 and of momentum into
 *                   directions 1-6, so the stored node keeps the computed mass and
 *                   momentum to within one binary16 spacing.
 *   LBM_F16S_SR     the LBM_F16S format, but the step rounds its stores stochastically:
 *                   each result x (scaled h) is stored as the nearest binary16 to x + d,
 *                   d uniform over one binary16 spacing of x (16-bit dither from a
 *                   counter-based hash of the node, the direction and a step counter
 *                   kept on the device), which rounds x up with probability equal to its
 *                   distance from the lower neighbour. Increments smaller than half a
 *                   spacing, which round-to-nearest drops, survive in expectation. Runs
 *                   are reproducible: the counter restarts at lbm_init_equilibrium and is
 *                   part of a saved state. lbm_adjoint returns LBM_EUNSUPPORTED for it.
 * lbm_get_f and lbm_get_f_box return f = w_i + h_i in FP64, lbm_set_f rounds f - w_i
 * to the stored format, and lbm_save_state copies the stored values as they are.
 * In LBM_F64_NATIVE every closure and model runs in FP64. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_F64_NATIVE = 3, LBM_F16S_SR = 4 } lbm_dtype;

enum { LBM_SOLID = 0, LBM_FLUID = 1, LBM_INLET = 2, LBM_OUTLET = 3 };
enum { LBM_PERIODIC_X = 1, LBM_PERIODIC_Y = 2, LBM_PERIODIC_Z = 4 };

/* Build a context for one geometry: validate the node types, build the tile map on
 * the GPU (Algorithm 1 of Sec. 3.1: tile_flag -> exclusive scan in z-y-x tile order ->
 * scatter of tileMap and nonEmptyTiles), build per-tile neighbour tables and node
 * masks, the work groups of the step kernel, and allocate the two population copies A
 * and B (Sec. 3.1, "two copies"). A copy stores the non-solid nodes only: the kept tiles
 * are cut into groups of consecutive tiles with at most 256 non-solid nodes, and each
 * group holds one 256-value block per direction (the nodes of a tile on consecutive
 * positions in slot order, the unused positions zero).
 *   node_type   nx*ny*nz bytes, dense; host memory if on_device == 0, else a device
 *               pointer. Values other than 0..3 give LBM_EINVAL.
 *   tile        must be 4 (the paper's a = 4), else LBM_EUNSUPPORTED.
 *   periodic    mask of LBM_PERIODIC_*; a periodic axis must be a multiple of 4
 *               (LBM_EINVAL). A non-periodic axis that is not a multiple of 4 is
 *               padded with solid nodes (Sec. 3.1).
 *   stream      cudaStream_t to queue work on (NULL = legacy default stream).
 *   out         receives the new context, or NULL on failure.
 * Limits: at most 2^31 / 64 kept tiles (2^31 node slots; per-node indices are 32-bit)
 * and at most 2^31 / 256 groups, else LBM_EUNSUPPORTED; device memory for two population
 * copies (LBM_ENOMEM).
 * The populations are not initialised: call lbm_init_equilibrium or lbm_set_f. */
lbm_status lbm_create(const uint8_t* node_type, int on_device, int nx, int ny, int nz, int tile,
                      lbm_dtype dtype, unsigned periodic, void* stream, lbm_ctx** out);

/* Release every device buffer of the context. NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last error of ctx ("" if none); with ctx == NULL, the last error of a
 * failed lbm_create in this thread. The string lives until the next call on ctx. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Change the stream later work is queued on. */
lbm_status lbm_set_stream(lbm_ctx* ctx, void* stream);

/* Relaxation time and boundary data (Eq. 2, Eq. 7; Sec. 2.2 boundary conditions).
 *   tau       LBGK relaxation time, must be > 1/2 and finite (else LBM_EINVAL).
 *   g         uniform body-force density (Guo forcing), 3 doubles; NULL = zero.
 *   g_field   optional per-node x component of the force density, nx*ny*nz doubles,
 *             dense; it replaces g[0] at every node. Host memory if
 *             g_field_on_device == 0, else a device pointer. NULL removes a field
 *             set earlier. The library keeps its own tile-major copy.
 *   u_in      velocity imposed at inlet nodes (3 doubles; NULL = zero).
 *   rho_out   density imposed at outlet nodes (> 0). */
lbm_status lbm_set_params(lbm_ctx* ctx, double tau, const double* g, const double* g_field,
                          int g_field_on_device, const double* u_in, double rho_out);

/* Collision model: the paper's variants (Sec. 2.2). equilibrium: LBM_EQ_QCOMPR (Eq. 3,
 * velocity Eq. 5; the default) or LBM_EQ_INCOMPR (Eq. 4, velocity Eq. 6: u = sum c f + F/2,
 * the reference density 1 in place of rho). collision: LBM_COLL_BGK (Eq. 2 / Eq. 7; the
 * default) or LBM_COLL_MRT (Eq. 8) in the D3Q19 moment basis of d'Humieres et al. (Phil.
 * Trans. R. Soc. A 360, 2002), equilibrium moments the projection of the equilibrium above
 * (so equal rates give LBGK), Guo forcing applied in moment space. rates: NULL for
 * d'Humieres et al.'s suggested D3Q19 rates, else 5 host doubles {s_e, s_eps, s_q, s_pi,
 * s_m} in (0, 2); the stress moments relax with 1/tau, the conserved ones with 1.
 * Applies to lbm_step, lbm_init_equilibrium and lbm_macroscopic (u = sum c f* - F/2 for
 * LBM_EQ_INCOMPR). Other models run their arithmetic in FP64 for the FP64 storage formats
 * and in FP32 on h = f - w for the others. LBM_EINVAL for an unknown model or a rate outside
 * (0, 2); lbm_adjoint supports only the default model. */
enum { LBM_EQ_QCOMPR = 0, LBM_EQ_INCOMPR = 1 };
enum { LBM_COLL_BGK = 0, LBM_COLL_MRT = 1 };
lbm_status lbm_set_model(lbm_ctx* ctx, int equilibrium, int collision, const double* rates);

/* Inlet/outlet scheme (Sec. 2.2). LBM_BC_EQUILIBRIUM (the default): inlet nodes take
 * f* = f^eq(rho, u_in), outlet nodes f* = f^eq(rho_out, u) (local equilibrium closures).
 * LBM_BC_ZOU_HE: the paper's Zou-He velocity inlet and constant-pressure outlet (Zou & He,
 * Phys. Fluids 9, 1997; D3Q19 with the transverse momentum correction of Hecht & Harting,
 * J. Stat. Mech. 2010): every inlet node lies on box face inlet_face and every outlet node
 * on outlet_face (0: x = 0, 1: x = nx - 1, 2: y = 0, 3: y = ny - 1, 4: z = 0,
 * 5: z = nz - 1), whose inward normal n fixes the unknown populations (c.n > 0); they are
 * completed so that the node has momentum rho u_in (u_in for the incompressible model) or
 * density rho_out with no tangential velocity, then the node collides as fluid. LBM_EINVAL
 * for an unknown scheme, a face outside 0..5 or on a periodic axis; lbm_adjoint supports
 * only the default. */
enum { LBM_BC_EQUILIBRIUM = 0, LBM_BC_ZOU_HE = 1 };
lbm_status lbm_set_bc(lbm_ctx* ctx, int scheme, int inlet_face, int outlet_face);

/* Moving wall (the lid of the cavity benchmark, Sec. 4.3): the box face `face` (0: x = -1,
 * 1: x = nx, 2: y = -1, 3: y = ny, 4: z = -1, 5: z = nz; its axis must not be periodic)
 * moves with velocity u (3 host doubles). A link whose source lies beyond that face
 * bounces back from the moving wall (Ladd, J. Fluid Mech. 271, 1994; wall density the
 * reference density 1): f_i(x) = f*_opp(i)(x) + 6 w_i (c_i . u). face = -1 removes it
 * (u may then be NULL). LBM_EINVAL for another face, a periodic axis or a non-finite u;
 * lbm_adjoint does not support a moving wall. */
lbm_status lbm_set_lid(lbm_ctx* ctx, int face, const double* u);

/* Set both population copies to the equilibrium f^eq(rho0, u0) of the context's model
 * (Eq. 3 by default) at every non-solid node. */
lbm_status lbm_init_equilibrium(lbm_ctx* ctx, double rho0, const double* u0);

/* Advance n >= 0 time steps: n launches of the fused step kernel, each reading the
 * current copy and writing the other, then swapping them (Sec. 3.1). Runs of 16 steps
 * are replayed from a CUDA graph captured on first use (and again after any call that
 * changes parameters, model, boundary scheme or lid). */
lbm_status lbm_step(lbm_ctx* ctx, int n);

/* The paper's calibration kernels (Sec. 4.1), which bound what the fused step can reach
 * with this data layout: LBM_KERNEL_PROPAGATE gathers with bounce-back exactly as the
 * step does and stores the gathered values without collision ("propagation only");
 * LBM_KERNEL_RW reads and writes each node's own 19 values ("read/write only", no
 * propagation). LBM_KERNEL_FULL is lbm_step. Same launch shape and A/B swap as lbm_step.
 * The populations afterwards are not a physical state for the calibration kinds. */
enum { LBM_KERNEL_FULL = 0, LBM_KERNEL_PROPAGATE = 1, LBM_KERNEL_RW = 2 };
lbm_status lbm_step_kernel(lbm_ctx* ctx, int kind, int n);

/* Density and velocity from the stored post-collision populations f*:
 * rho = sum_i f*_i, u = (sum_i c_i f*_i - F/2) / rho (Eq. 5 with the half-force shift of
 * Guo forcing; Eq. 6, without the division, for LBM_EQ_INCOMPR); 0 at solid nodes.
 * rho: nx*ny*nz values, u: 3*nx*ny*nz values, dense, double if out_f64 else float;
 * device pointers if on_device, else host. */
lbm_status lbm_macroscopic(lbm_ctx* ctx, void* rho, void* u, int out_f64, int on_device);

/* Global invariants over non-solid nodes, accumulated in FP64 with warp shuffles and a
 * fixed-order second pass (deterministic): *mass = sum f*, momentum = sum (sum c f* - F/2).
 * Host outputs. Returns LBM_ENONFINITE if the mass is NaN or Inf. */
lbm_status lbm_reduce(lbm_ctx* ctx, double* mass, double* momentum);

/* Export the populations of the box [x0, x0+bx) x [y0, y0+by) x [z0, z0+bz) as FP64
 * [19][bz][by][bx] into host memory `out` (for FP16S, f = w + h). Coordinates wrap on
 * periodic axes; nodes that are solid, padding or outside the domain read NaN. */
lbm_status lbm_get_f_box(lbm_ctx* ctx, int x0, int y0, int z0, int bx, int by, int bz, double* out);

/* Whole-domain export / import of the current populations, dense FP64
 * [19][nz][ny][nx] host arrays; solid entries are ignored on import and NaN on export. */
lbm_status lbm_get_f(lbm_ctx* ctx, double* f_dense);
lbm_status lbm_set_f(lbm_ctx* ctx, const double* f_dense);

/* Gradient of an outlet-flux loss by a hand-written discrete adjoint of the step (the
 * paper has no adjoint; the forward map is the step of Sec. 3.4 / Eq. 7). From the
 * current state s_0: T steps forward (the context ends in s_T, as after lbm_step(T)),
 *   L = mean over non-solid nodes of the plane x = plane_x of u_x(s_T),
 *       u_x = (sum_i c_ix f*_i - F_x/2) / rho,
 * and, if dL_dg or dL_dtau is not NULL, the reverse sweep: a checkpoint is kept every
 * ckpt_every steps, each segment is recomputed from its checkpoint and T adjoint-step
 * kernels run backwards.
 *   loss      host, receives L (0 if the plane has no non-solid node).
 *   dL_dg     nx*ny*nz doubles, dense: dL/dF_x per node, F_x being the per-node x force
 *             (the field of lbm_set_params, or g[0] everywhere); 0 at solid nodes.
 *             Device pointer if dL_dg_on_device, else host. May be NULL.
 *   dL_dtau   host, receives dL/dtau. May be NULL.
 * Gradients accumulate in FP64; the adjoint arithmetic runs in the storage's arithmetic
 * precision (FP64 for LBM_F64, FP32 otherwise). Device memory: (ceil(T/ckpt_every) +
 * min(ckpt_every, T)) population copies plus two adjoint copies; if it cannot be
 * allocated the call returns LBM_ENOMEM before any work and the state is unchanged.
 * LBM_EUNSUPPORTED for a context of format LBM_F16S_SR (its recompute would not
 * reproduce the forward's random rounding without storing the counter per segment),
 * with a model other than quasi-compressible LBGK, a moving wall or Zou-He boundaries. */
lbm_status lbm_adjoint(lbm_ctx* ctx, int T, int ckpt_every, int plane_x, double* loss, double* dL_dg,
                       int dL_dg_on_device, double* dL_dtau);

/* Tile structures (Sec. 3.1): tile_map has ceil(nx/4)*ceil(ny/4)*ceil(nz/4) int32 entries
 * (rank of the tile among the kept tiles, or -1), non_empty has *n_tiles uint32 linear tile
 * indices t = tx + Tx (ty + Ty tz) in discovery order. Either array may be NULL. Host. */
lbm_status lbm_get_tiles(lbm_ctx* ctx, int32_t* tile_map, uint32_t* non_empty, int64_t* n_tiles);

/* Sizes: n_tiles kept, n_nonsolid nodes, bytes of one population copy (19 * 256 values per
 * group, unused positions included). Any may be NULL. */
lbm_status lbm_get_info(lbm_ctx* ctx, int64_t* n_tiles, int64_t* n_nonsolid, int64_t* copy_bytes);

/* Copy the current state (the populations and, for LBM_F16S_SR, the step counter of the
 * rounding) to a host blob, or back.
 * lbm_save_state with blob == NULL stores the size in *nbytes. The blob carries a
 * checksum and a hash of the geometry; loading a blob of another geometry, dtype or
 * with a bad checksum gives LBM_ESTATE. */
lbm_status lbm_save_state(lbm_ctx* ctx, void* blob, size_t* nbytes);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* blob, size_t nbytes);

/* ------------------------------------------------------------------------------------
 * Domain decomposition into z-slabs with a halo exchange (the paper names multi-GPU
 * execution as future work, Sec. 5; the step itself is unchanged, Sec. 3.4). Each rank
 * owns a contiguous range of tile planes along z, the outermost axis of the tile order
 * (Sec. 3.1), so its tiles and its ghost tiles are contiguous rank ranges. Before every
 * step the populations that cross a cut -- the five directions with c_z = +1 or -1 --
 * of the boundary tiles are copied into the neighbouring slab's ghost plane; mass and
 * momentum are summed over ranks in FP64. The transport between ranks is the caller's
 * (the Python binding uses torch.distributed). */

/* Split the tile planes along z into nranks contiguous slabs of about equal numbers of
 * non-solid nodes. Host only, no GPU needed.
 *   node_type    host, nx*ny*nz bytes (the whole domain).
 *   plane_begin  host, nranks + 1 ints: rank r owns tile planes [plane_begin[r],
 *                plane_begin[r+1]); plane_begin[0] = 0, plane_begin[nranks] = ceil(nz/4).
 * LBM_EINVAL unless 1 <= nranks <= ceil(nz/4); every slab gets at least one plane. */
lbm_status lbm_partition_z(const uint8_t* node_type, int nx, int ny, int nz, int nranks, int* plane_begin);

/* The node types of a slab's box: its own tile planes [plane_begin, plane_end) plus one
 * ghost tile plane below and above where the domain continues there (always on a
 * periodic z axis, else not at the domain's ends); no ghost planes if the slab is the
 * whole domain. Host only, no GPU needed.
 *   sub          host, nx*ny*(*nz_sub) bytes, or NULL to ask only for the sizes; padding
 *                nodes beyond nz are solid.
 *   nz_sub       receives the box's z extent (4 per tile plane).
 *   ghost_lo/hi  receive 1 for a ghost plane at the bottom / top of the box, else 0
 *                (either may be NULL).
 * LBM_EINVAL for an empty or out-of-range plane range or a periodic z axis that is not a
 * multiple of 4. */
lbm_status lbm_slab_geometry(const uint8_t* node_type, int nx, int ny, int nz, unsigned periodic, int plane_begin,
                             int plane_end, uint8_t* sub, int* nz_sub, int* ghost_lo, int* ghost_hi);

/* A context for one slab: lbm_create on the slab's box (lbm_slab_geometry), periodic in
 * x and y as given, its ghost planes standing for the rest of the domain along z. The
 * step, lbm_reduce and lbm_macroscopic cover the own tiles only; lbm_init_equilibrium,
 * lbm_set_f / lbm_get_f / lbm_get_f_box and lbm_save_state cover the whole box, in box
 * coordinates (box z = 0 is global node z = 4 (plane_begin - ghost_lo), wrapped on a
 * periodic axis). lbm_get_info counts the own non-solid nodes. lbm_adjoint returns
 * LBM_EUNSUPPORTED. A slab that is the whole domain is a plain lbm_create context.
 *   node_type    host, the whole domain's nx*ny*nz node types.
 * Other arguments and errors as lbm_create and lbm_slab_geometry. */
lbm_status lbm_create_slab(const uint8_t* node_type, int nx, int ny, int nz, int tile, lbm_dtype dtype,
                           unsigned periodic, int plane_begin, int plane_end, void* stream, lbm_ctx** out);

/* Halo of a slab context, on its current population copy (call between steps).
 *   side  0: the bottom of the box, 1: the top.
 *   lbm_halo_pack copies the populations the neighbouring slab on that side reads from
 *   this slab's boundary plane (side 0: the lowest own plane, directions with c_z = -1;
 *   side 1: the highest, c_z = +1) into buf, [direction][tile][64] in the stored format
 *   (NaN in the solid and padding slots);
 *   lbm_halo_unpack copies such a buffer, packed by that neighbour on the opposite side,
 *   into the ghost plane on this side. The two planes hold the same kept tiles in the
 *   same order, since both slabs were cut from the same geometry.
 *   lbm_halo_bytes gives the size of the buffer pack (pack = 1) or unpack (pack = 0)
 *   uses on that side: 5 * 64 * (bytes per value) per tile of the plane.
 *   buf   device pointer, on the context's stream; the copy kernel is queued, not awaited.
 * LBM_ESTATE if the box has no ghost plane on that side or no state is set. */
lbm_status lbm_halo_bytes(lbm_ctx* ctx, int side, int pack, size_t* bytes);
lbm_status lbm_halo_pack(lbm_ctx* ctx, int side, void* buf);
lbm_status lbm_halo_unpack(lbm_ctx* ctx, int side, const void* buf);

/* Allocation-free tile-map builder. The paper has no counterpart to this entry point.
 * It is for callers that cannot call cudaMalloc -- code running under a framework whose
 * caching allocator has reserved the device memory, or hosts that forbid allocation
 * after start-up -- and that already own their input and output buffers.
 * It computes what lbm_create builds (tileMap and nonEmptyTiles, bit for bit) but takes
 * its temporary storage (one flag byte per tile, scan block sums, the count and an
 * error flag) from one static device array of 4,227,584 bytes that every GPU loading
 * this library holds until the process exits; it calls no cudaMalloc or cudaFree.
 *   node_type  device pointer, nx*ny*nz bytes, dense, values 0..3.
 *   tile_map   device pointer, ceil(nx/4)*ceil(ny/4)*ceil(nz/4) int32 (written in full).
 *   non_empty  device pointer with room for as many uint32 as tile_map has entries; the
 *              first *n_tiles are written.
 *   n_tiles    host pointer; receives the number of kept tiles.
 *   stream     cudaStream_t for the work; the call synchronises it before returning.
 * Limits and errors: at most LBM_NOALLOC_MAX_TILES tiles in the tile grid (e.g. a
 * 1024 x 512 x 512 box); larger grids give LBM_EUNSUPPORTED before any device work.
 * The library cannot check the extent of the three device buffers: a host pointer or
 * a buffer smaller than stated above is read or written out of bounds (the Python
 * binding checks both before the call). NULL pointers or dimensions < 1 give LBM_EINVAL, node types outside 0..3 give
 * LBM_EINVAL after the kernels ran, CUDA failures LBM_ECUDA. There is no message string.
 * The first call on each device looks up the array's device address (with that device
 * current); make that first call before any stream capture. All calls share the one
 * array, so calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must not be issued. */
#define LBM_NOALLOC_MAX_TILES (1 << 22)
lbm_status lbm_build_tiles_noalloc(const uint8_t* node_type, int nx, int ny, int nz, int32_t* tile_map,
                                   uint32_t* non_empty, int64_t* n_tiles, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
