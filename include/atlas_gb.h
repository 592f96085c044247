/*
 * atlas_gb.h -- C ABI of libatlasgb.so: median-dual finite-volume nabla
 * operators (gradient, divergence, Laplacian, the adjoints of gradient and
 * divergence, curl and the gradient of a tangent vector field) on multi-level
 * fields over the octahedral reduced Gaussian grid (also the regular Gaussian
 * grid and regional grids of map projections), with FP64 conservation sums,
 * band partitions and grid-to-grid remapping, computed by CUDA kernels on
 * one GB300 (sm_103a).
 *
 * The paper (ESCAPE D2.3, the Atlas release) describes the workflow
 * Grid -> Mesh -> FunctionSpace -> Field (Sec. 2.3, Fig. 1 and Fig. 2), says
 * that Atlas supplies gradient, divergence, curl and Laplacian operators
 * on it (Sec. 2.3), exposes its C++ objects through C interfaces holding raw
 * pointers (Sec. 4.1, Fig. 3), keeps Fields in host and device memory that
 * are synchronised explicitly (Sec. 4.2, Listings 3 and 4), and brackets use
 * of the library with initialise/finalise (Sec. 3.5, Listings 1 and 2).  The
 * calls below follow that shape.
 *
 * Conventions (all calls):
 *   - Return 0 on success or a negative ATLAS_E* code; atlas_last_error()
 *     then returns a message (thread-local, valid until the next call on the
 *     same thread).  No C++ exception crosses this interface.
 *   - Handles (atlas_grid_t, atlas_mesh_t, atlas_fvm_t, atlas_batch_t,
 *     atlas_part_t, atlas_remap_t) are owned by the library and released by
 *     the matching *_destroy call.  A mesh keeps a reference to its grid, an
 *     fvm to its mesh, a batch or partition to its fvms, a remap to its mesh
 *     and target grid: destroy in reverse order of creation (a destroy that
 *     would break a reference does nothing and leaves an ATLAS_ESTATE
 *     message in atlas_last_error).
 *   - Field pointers are DEVICE pointers owned by the caller (for example
 *     torch tensors); the library never frees them.  A field is stored
 *     field[node][level]: node i, level k at element offset i*ld + k, with
 *     nlev >= 0 levels and leading dimension max(nlev, 1) <= ld <= 2^31 - 1
 *     (elements; a larger ld is refused with ATLAS_EINVAL).  When
 *     ld is a multiple of the vector width (16 bytes: 4 F32, 2 F64, 8 BF16
 *     levels) outputs are written in whole vectors and the padding levels
 *     from nlev to the end of the row's last vector are set to zero; all
 *     later levels below ld are never written.  Nodes are numbered row by
 *     row from north to south, and within a row by increasing longitude
 *     starting at 0 (regional grids: by rows of decreasing y, then x).
 *   - dtype selects the storage type of every field argument of the call:
 *     ATLAS_F32 (float, FP32 arithmetic), ATLAS_F64 (double, FP64
 *     arithmetic) or ATLAS_BF16 (bfloat16 storage, FP32 arithmetic).
 *     Geometry is FP64 on the host and converted once per dtype.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Operator
 *     calls only enqueue work and return; a kernel that fails to launch is
 *     reported as ATLAS_ECUDA, faults during execution surface at the
 *     caller's next synchronisation.  The first operator call of a kind on an
 *     fvm builds and uploads that operator's tables synchronously (or call
 *     atlas_fvm_prepare first); keep first calls out of CUDA-graph capture.
 *   - Pointers must be aligned to the element size; the vectorised paths
 *     additionally need 16-byte aligned rows (ld a multiple of 16/sizeof),
 *     and fall back to element-wise loads otherwise.
 *   - Input and output fields of one call must not overlap.
 *   - Calls may come from several host threads at once.  Builds of distinct
 *     objects run concurrently; the tables that one fvm (or remap) builds on
 *     first use are built once, under that object's lock, whichever thread
 *     asks first.  A handle must not be destroyed while another thread is
 *     still inside a call that uses it.
 *   - No call ever computes on the CPU: without a CUDA device every operator
 *     call fails with ATLAS_ECUDA.
 *   - Bounds-checked build (the library compiled with -DATLASGB_BOUNDSCHECK,
 *     a debugging aid): every kernel checks each index it takes from a table
 *     (neighbour ids, CSR row ranges, edge ids, staged slots, copy ranges)
 *     against the buffers of its launch, skips an access that would leave
 *     them and records the first such index in a device word; every
 *     operator, batch and remap call then waits for its stream and returns
 *     ATLAS_EBOUNDS, with the kernel's check code and the index in
 *     atlas_last_error().  Tables are validated on the host before upload
 *     (atlas_fvm_load refuses inconsistent connectivity), so a library
 *     table never trips a check; the checks guard the kernels' own index
 *     arithmetic.  atlas_info() names the build.
 */
#ifndef ATLAS_GB_H
#define ATLAS_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct atlas_grid_s* atlas_grid_t;
typedef struct atlas_mesh_s* atlas_mesh_t;
typedef struct atlas_fvm_s* atlas_fvm_t;
typedef struct atlas_batch_s* atlas_batch_t;
typedef struct atlas_remap_s* atlas_remap_t;

typedef enum { ATLAS_F32 = 0, ATLAS_F64 = 1, ATLAS_BF16 = 2 } atlas_dtype;

enum {
  ATLAS_OK = 0,
  ATLAS_EINVAL = -1,  /* invalid argument (null pointer, size, ld < nlev, ...) */
  ATLAS_ENOMEM = -2,  /* host or device allocation failed */
  ATLAS_ECUDA = -3,   /* CUDA runtime error, or no CUDA device */
  ATLAS_EALIGN = -4,  /* pointer not aligned to its element size */
  ATLAS_EDTYPE = -5,  /* unsupported dtype */
  ATLAS_ESTATE = -6,  /* handle in the wrong state (destroyed, wrong device) */
  ATLAS_EBOUNDS = -7  /* bounds-checked build only: a kernel met a table index
                         outside its buffers (the access was skipped) */
};

/* Operator identifiers (atlas_fvm_prepare masks use 1 << op). */
enum {
  ATLAS_OP_GRADIENT = 0,
  ATLAS_OP_DIVERGENCE = 1,
  ATLAS_OP_GRADIENT_ADJOINT = 2,
  ATLAS_OP_DIVERGENCE_ADJOINT = 3,
  ATLAS_OP_LAPLACIAN = 4,
  ATLAS_OP_CURL = 5,
  ATLAS_OP_VECTOR_GRADIENT = 6,
  ATLAS_OP_CURL_ADJOINT = 7
};

/* Map projections of regional grids (atlas_grid_regional). */
enum {
  ATLAS_PROJ_ROTATED_LONLAT = 0,
  ATLAS_PROJ_MERCATOR = 1,
  ATLAS_PROJ_LAMBERT_CONFORMAL = 2,
  ATLAS_PROJ_POLAR_STEREOGRAPHIC = 3
};

/* ---------------------------------------------------------------------- */
/* Library lifecycle (paper Sec. 3.5, Listings 1-2: initialise/finalise). */
/* Both are idempotent and optional; finalize releases nothing the caller  */
/* still holds.                                                            */
/* ---------------------------------------------------------------------- */
int atlas_init(void);
int atlas_finalize(void);
/* Version string and a one-line feature report (GPU name, sm, build).   */
const char* atlas_version(void);
const char* atlas_info(void);
const char* atlas_last_error(void);

/* ---------------------------------------------------------------------- */
/* Grid (paper Sec. 2.3: a grid is only a set of 2-D points, given ahead; */
/* the O<N> octahedral grid is named in Sec. 4.3, Fig. 4).                 */
/* ---------------------------------------------------------------------- */
/* Octahedral reduced Gaussian grid O<N>, 1 <= N <= 8000: 2N Gaussian      */
/* latitudes (roots of the Legendre polynomial P_2N, north to south); row  */
/* r holds 4i+16 equally spaced longitudes starting at 0, i = r+1 for      */
/* r < N and 2N-r otherwise; 4N^2+36N points.                              */
int atlas_grid_octahedral(int N, atlas_grid_t* out);
/* Views into library-owned arrays, valid until atlas_grid_destroy:        */
/* nnodes, nlat = 2N, pl[nlat] points per row, lonlat[nnodes][2]           */
/* (longitude, latitude in radians), lat[nlat] row latitudes (radians).    */
/* Any output pointer may be NULL.                                         */
int atlas_grid_info(atlas_grid_t g, int64_t* nnodes, int* nlat, const int32_t** pl,
                    const double** lonlat, const double** lat);
/* Regular (full) Gaussian grid F<N>, 1 <= N <= 8000 (paper Sec. 4.3,     */
/* Fig. 4 and 6: the coarse "F8" grid): the 2N Gaussian latitudes of O<N>, */
/* each with 4N equally spaced longitudes from 0; 8N^2 points, same node   */
/* order.  A remapping target, and a grid for meshes and operators like    */
/* O<N> (the zipper then meets equal rows on every band; pole edges join  */
/* node j to j + 2N on the first and last row).                            */
int atlas_grid_regular_gaussian(int N, atlas_grid_t* out);

/* Regional (limited-area) grids (paper Sec. 2.2.3 and Sec. 5: Atlas meshes */
/* the regional grids of limited-area models; operators that account for   */
/* the projection are the follow-up work named there).  A rectangle of a   */
/* map projection's plane with nx >= 2 points per row and ny >= 2 rows,    */
/* nx * ny <= 2^28:                                                        */
/*   x_j = xmin + j (xmax - xmin)/(nx - 1),  y_r = ymax - r (ymax - ymin)/(ny - 1), */
/* node id r nx + j (the first row has the largest y).  params[8] =        */
/* {xmin, xmax, ymin, ymax, p4, p5, p6, p7}:                               */
/*   ATLAS_PROJ_ROTATED_LONLAT: x, y are rotated longitude and latitude in */
/*     degrees, |y| < 90, xmax - xmin < 360; (p4, p5) = longitude and      */
/*     latitude of the rotated south pole in degrees (GRIB convention; (0, */
/*     -90) is the plain lon-lat grid); p6, p7 unused.                     */
/*   ATLAS_PROJ_MERCATOR: x, y in metres; p4 = radius of the projection    */
/*     sphere (metres), p5 = central longitude (degrees); |y|/p4 <= 7.     */
/*   ATLAS_PROJ_LAMBERT_CONFORMAL: tangent cone; x, y in metres; p4 =      */
/*     radius, p5 = central longitude, p6 = tangent latitude (degrees,     */
/*     0 < |p6| < 90); the domain must not hold the pole or cross the cut  */
/*     opposite the central longitude.                                     */
/*   ATLAS_PROJ_POLAR_STEREOGRAPHIC: plane tangent at the pole p6 = 90 or   */
/*     -90, projected from the opposite pole; x, y in metres; p4 = radius, */
/*     p5 = the longitude along -y from the north pole (+y from the south  */
/*     pole); the domain may hold its pole.                                */
/* Every point must stay more than about 0.06 degrees from a pole of the  */
/* projection.  EINVAL (with the reason in atlas_last_error) otherwise.    */
/* atlas_grid_info then reports nlat = ny rows of nx points and lat[r] =   */
/* the latitude of row r's first point.                                   */
int atlas_grid_regional(int projection, int nx, int ny, const double* params, atlas_grid_t* out);
/* Regional grids only (EINVAL otherwise): projection, nx, ny, the plane   */
/* coordinates xy[nnodes][2] on the unit sphere (radians, or metres over   */
/* the projection radius) and the scale factors scale[nnodes][2] = (h_x,   */
/* h_y): a plane step dx is a true distance R h_x dx on a sphere of radius */
/* R (rotated lon-lat: (cos y, 1); conformal projections: 1/m, the inverse map */
/* factor, in both directions).                                            */
int atlas_grid_regional_info(atlas_grid_t g, int* projection, int* nx, int* ny, const double** xy,
                             const double** scale);
void atlas_grid_destroy(atlas_grid_t g);

/* ---------------------------------------------------------------------- */
/* Mesh (paper Sec. 2.3: connectivity of elements, edges and nodes).       */
/* ---------------------------------------------------------------------- */
/* A regional grid is meshed two triangles per quad: quad (r, j) with a =  */
/* r nx + j is split along (a, a+nx+1) into {a, a+nx+1, a+1} and {a, a+nx, */
/* a+nx+1} (counter-clockwise in the plane); 2 (nx-1)(ny-1) triangles,     */
/* 3 nx ny - 2 nx - 2 ny + 1 edges, none of them pole edges.               */
/* Zipper triangulation of every pair of adjacent rows (advance on the row */
/* whose next longitude is smaller; on a tie the row with fewer points,    */
/* between equal rows the northern one), plus pole edges joining node j to */
/* j + n/2 on the first and last row.  Edges are (a, b) with a < b, sorted */
/* by (a, b); 4N^2+36N nodes give 2V-40 triangles and 3V-20 edges (F<N>: */
/* 8N^2 nodes, 2V-8N triangles, 3V-4N edges).                               */
int atlas_mesh_build(atlas_grid_t g, atlas_mesh_t* out);
/* Views valid until atlas_mesh_destroy: e2n[E][2], is_pole[E],            */
/* n2e_ptr[V+1], n2e[2E] (ascending edge ids per node), n2e_sign[2E]       */
/* (+1 where the node is the edge's a, -1 where it is b), tri[T][3].       */
int atlas_mesh_info(atlas_mesh_t m, int64_t* nedges, int64_t* ntri, const int32_t** e2n,
                    const uint8_t** is_pole, const int32_t** n2e_ptr, const int32_t** n2e,
                    const int8_t** n2e_sign, const int32_t** tri);
void atlas_mesh_destroy(atlas_mesh_t m);

/* ---------------------------------------------------------------------- */
/* Finite-volume geometry (the FunctionSpace of nodes, paper Sec. 2.3).    */
/* ---------------------------------------------------------------------- */
/* Median dual in the (lon, lat) plane with radius R (metres): every node  */
/* owns the polygon of its side midpoints and triangle centroids, extended */
/* to the pole on the first and last rows.  V_i = R^2 * integral of        */
/* cos(lat) over the cell; S_e = R (dlat, -dlon) integrated along the dual */
/* face of edge e from cell a into cell b; pole edges carry the pole       */
/* segment normal (0, +-2 pi R / n).  Everything is FP64 on the host; the  */
/* call also records the current CUDA device, on which every operator of  */
/* this fvm must then run, and ends with the checks of atlas_fvm_check     */
/* (EINVAL if the geometry came out inconsistent).                         */
int atlas_fvm_build_dual(atlas_mesh_t m, double radius, atlas_fvm_t* out);
/* Host FP64 views valid until atlas_fvm_destroy: V[nnodes], S[E][2],      */
/* coslat[nnodes], pole_nphi[nnodes] (phi-normal of the pole segment).     */
int atlas_fvm_info(atlas_fvm_t f, const double** V, const double** S, const double** coslat,
                   const double** pole_nphi);
/* The dual of a regional grid lies in the projection plane: S_e = R times */
/* the integrated plane normal of the face of edge e (a to b), area[i] =   */
/* R^2 times the plane area of cell i (a third of each adjacent triangle), */
/* Sb[E][2] = R times the outward plane normal of a boundary edge (0 for  */
/* interior edges), V_i = h_x,i h_y,i area_i, pole_nphi = 0 and coslat the */
/* cosine of the node latitude.  Operators on it use face values          */
/* (f_i + f_j)/2 on interior faces and (5 f_i + f_j)/6 on boundary half    */
/* edges (exact for fields linear in the plane), the scale factors at the */
/* nodes, and give vector components along the grid's x and y directions: */
/*   gradient  (h_x^-1 d/dx, h_y^-1 d/dy) f                               */
/*   divergence (h_x h_y)^-1 [d(h_y u)/dx + d(h_x v)/dy]                  */
/*   curl       (h_x h_y)^-1 [d(h_y v)/dx - d(h_x u)/dy]                  */
/* with the Laplacian = divergence(gradient), the adjoints the transposes */
/* and the vector gradient the gradient of each component.  The           */
/* edge-based two-pass calls refuse a regional fvm (EINVAL).               */
/* Regional fvm only (EINVAL otherwise): area[nnodes] and Sb[E][2].         */
int atlas_fvm_regional_info(atlas_fvm_t f, const double** area, const double** Sb);

/* Volume-weighted sums in FP64 (the global conservation sums; the paper */
/* gives no counterpart, they check the operators of Sec. 2.3): for every  */
/* level k, out[k] = sum over nodes i = node0 .. node0+count-1 of          */
/* V_i x[(i - node0) ld + k], where x points at the row of node node0 (a  */
/* partition's own rows: sum its part, then add the parts across ranks).  */
/* Of the divergence and the curl the sum over the whole sphere vanishes   */
/* (conservation).  x is F32, F64 or BF16 with the usual layout rules; out */
/* is a device array of nlev doubles; ws a device workspace of            */
/* atlas_fvm_integral_workspace_bytes(f, nlev) bytes, 8-byte aligned, used */
/* by this call only.  Deterministic: FP64 partial sums of fixed node     */
/* blocks (four interleaved accumulators each), added in block order; no  */
/* atomics.  Enqueued on stream.                                           */
size_t atlas_fvm_integral_workspace_bytes(atlas_fvm_t f, int nlev);
int atlas_fvm_integral(atlas_fvm_t f, const void* x, int64_t node0, int64_t count, int nlev, int64_t ld,
                       atlas_dtype dtype, double* out, void* ws, size_t ws_bytes, void* stream);
/* Consistency check of an fvm's host geometry (host only, O(E)): the      */
/* node->edge CSR holds every edge exactly twice, at its first node with  */
/* sign +1 and at its second with -1; edge ends are ordered and in range;  */
/* volumes are positive; and every dual cell closes: the sum of its        */
/* outward face normals (pole faces at both ends; half of each boundary   */
/* edge's outward normal on regional grids) is at most 1e-12 of the sum of */
/* their absolute values.  worst_closure (may be NULL) receives the        */
/* largest such ratio.  EINVAL naming the first bad node otherwise.        */
int atlas_fvm_check(atlas_fvm_t f, double* worst_closure);
/* Geometry cache.  atlas_fvm_save writes the fvm's host grid, mesh and   */
/* dual (FP64, bit for bit, with a checksum) to the file path;             */
/* atlas_fvm_load reads one back as three new handles (grid, mesh, fvm,   */
/* linked as if built by atlas_grid_* / atlas_mesh_build /                 */
/* atlas_fvm_build_dual, and destroyed the same way), after the checks of  */
/* atlas_fvm_check.  EINVAL with the reason for an unreadable, truncated,  */
/* corrupted or inconsistent file.  Host only.                             */
int atlas_fvm_save(atlas_fvm_t f, const char* path);
/* The sphere radius the fvm's dual was built with (metres).               */
int atlas_fvm_radius(atlas_fvm_t f, double* radius);
int atlas_fvm_load(const char* path, atlas_grid_t* grid, atlas_mesh_t* mesh, atlas_fvm_t* fvm);
/* Testing hook: let the next `after` device allocations of the library    */
/* succeed and fail every one after them (as out of memory) until called   */
/* again with -1 (the default: never fail).  Calls that need an            */
/* allocation then return ATLAS_ENOMEM and leave no partial tables behind. */
/* Process-wide.                                                           */
int atlas_debug_fail_allocations(int after);
/* Build and upload the tables of the operators in op_mask (bits 1<<op)    */
/* for the dtypes in dtype_mask (bits 1<<dtype), with the edge-based       */
/* tables of the gradient and divergence on global grids.  Synchronous.    */
int atlas_fvm_prepare(atlas_fvm_t f, unsigned op_mask, unsigned dtype_mask);
/* Launch shape of the node-stencil kernels for one operator and storage  */
/* dtype (atlas_dtype, or -1 for all three; each starts from a measured    */
/* default): levels per                                                    */
/* thread (vec: 1, 2, 4 or 8; 0 = default for the dtype), CSR entries per */
/* load batch (batch: 3 or 6), threads per block (64..512, multiple of    */
/* 32), blocks per SM (1..32) and tile_passes (1..4096): each block walks */
/* tiles of tile_passes * threads consecutive (node, level-vector) items, */
/* 1 being a plain grid-stride loop (default).  Tiles apply to BF16       */
/* fields and to the F32 Laplacian; the other F32 and F64 kernels always  */
/* run a grid-stride loop.  Any zero field keeps the current value;       */
/* results are bitwise identical for every shape.                          */
int atlas_fvm_set_launch(atlas_fvm_t f, int op, int dtype, int vec, int batch, int threads, int blocks_per_sm,
                         int tile_passes);
/* Shared-memory node-group kernels (FP32 and BF16 fields; F64 always runs */
/* per node).  Every grid row is cut into tiles of up to groups_per_tile  */
/* groups of four consecutive nodes; a producer warp copies the node rows */
/* a tile reads (its own and their neighbours, a few runs of consecutive  */
/* ids) into shared memory with TMA bulk copies, up to four tiles ahead,  */
/* and the consumer warps (one per group, or two per group with two nodes */
/* each) walk their nodes' stencil rows from shared memory.  They apply   */
/* where the field pointers are 16-byte aligned, ld * element size is a   */
/* multiple of 16, two stages of a tile's rows fit in shared memory (at   */
/* O1280 x 137 FP32 with ld 140: every operator) and the launch is made   */
/* of whole tiles (whole grids, partitions of whole rows); elsewhere the  */
/* per-node kernels run, with bitwise identical results.                  */
/* enable: 1 (default) uses them for the FP32 and BF16 operators, the     */
/* one-ring operators only on fields of more than 80 levels (FP32) or 96  */
/* (BF16): their table work per tile does not shrink with the levels, and */
/* below that the per-node kernels measured as fast or faster; 2 uses     */
/* them wherever they apply; 0 per-node kernels only; -1 keeps.            */
/* blocks_per_sm: 1 or 2 blocks per SM at most (fewer when shared memory  */
/* or registers are short; 0 keeps; default 1: one block holding up to    */
/* four stages measured faster than two blocks of two).                   */
/* groups_per_tile: 1..15 (0 keeps).  Defaults: FP32 10, the Laplacian  */
/* 12; BF16 11, the Laplacian and the one-input operators 15.  More than */
/* 11 run only where the kernel fits in 128 registers (the Laplacian, the */
/* BF16 one-input operators); with two warps per group at most 7 run.     */
/* Elsewhere the call falls back to the per-node kernel.  A change        */
/* rebuilds the operator's tile tables at its next call.                  */
/* nodes_per_warp: 4 (one consumer warp per group) or 2 (two warps per    */
/* group, each walking two of its nodes: twice the warps per block); 0    */
/* keeps; default 4.  With one warp per group the tables store the groups */
/* whose union of stencil rows matches the operator's pattern in union    */
/* form (atlas_fvm_tile_union_groups): each distinct neighbour row is      */
/* read once for the group's four nodes.  A change rebuilds the tables.   */
/* rows_per_tile: 1..3 grid rows a tile spans (0 keeps; default 2 for     */
/* FP32 fields, 1 for BF16): tile                                          */
/* k of a run of that many consecutive rows holds groups k * G .. k * G + */
/* G - 1 of each row, G = groups_per_tile / rows_per_tile.  The rows above */
/* and below are then staged once for several output rows (a two-ring     */
/* tile of two rows stages six grid rows, not ten).  Launches must cover  */
/* whole runs of rows: the rows of a run that a launch cuts (a partition */
/* boundary) run on the per-node kernel, with identical results.  A run  */
/* whose tile would need more than 16 copy runs (rows near the poles) is  */
/* tiled row by row.  A change rebuilds the tables.                        */
/* dtype -1 sets all three dtypes.  Host only; takes effect at the next   */
/* operator call.                                                          */
int atlas_fvm_set_group(atlas_fvm_t f, int op, int dtype, int enable, int blocks_per_sm, int groups_per_tile,
                        int nodes_per_warp, int rows_per_tile);
/* Launch shape the node-group kernel of one operator takes on fields of   */
/* nlev levels and leading dimension ld (16-byte aligned pointers          */
/* assumed): blocks per SM, pipeline stages per block, dynamic shared      */
/* memory per block in bytes, and the most node rows a tile stages; all 0  */
/* when the operator runs per node for these sizes (F64, unaligned rows,  */
/* tiles too large for shared memory).  Builds the operator's tables.      */
int atlas_fvm_tile_info(atlas_fvm_t f, int op, int dtype, int nlev, int64_t ld, int* blocks_per_sm, int* stages,
                        int64_t* smem_bytes, int64_t* max_rows);
/* FP64 rate probe (the FP64 operators are bound by GB300's FP64 pipe):    */
/* launches blocks x threads threads (threads a multiple of 32, <= 256),   */
/* each running 8 independent chains of iters dependent FP64 fused        */
/* multiply-adds, 16 * iters flops per thread, and stores one double per  */
/* thread in out (device, blocks * threads doubles).  The caller times it */
/* (CUDA events on the stream) to measure the FP64 rate the FP64 roofline */
/* is quoted against.                                                      */
int atlas_fp64_fma_rate_kernel(double* out, int blocks, int threads, int64_t iters, void* stream);
/* The node-group kernels bound every wait on their pipeline barriers      */
/* (about a second); a kernel that gives up records a code in a device     */
/* error word and returns, its outputs then incomplete.  This call copies  */
/* that word (synchronously: it waits for the device) into *code, 0 when   */
/* no kernel gave up, and with clear != 0 resets it.  Codes (bits): 1 a    */
/* consumer warp gave up waiting for a tile, 2 the producer gave up        */
/* waiting for a free stage, 4 copies were still in flight when the        */
/* producer left.                                                          */
int atlas_kernel_status(unsigned* code, int clear);
/* Testing hook: with on != 0 the following node-group launches make their */
/* consumer warps wait on a barrier that nothing completes, with a limit of */
/* a few milliseconds, so that the time-out path runs (code 1); 0 restores  */
/* normal launches.  No GPU fault and no hang is involved.                  */
int atlas_debug_tile_hang(int on);
/* Tuning hook: the consumer warps of the node-group kernels wait for a    */
/* tile's copies with mbarrier try-waits that may suspend the thread for   */
/* up to ns nanoseconds each (0, the default: the hardware's own short    */
/* suspension).  Results do not depend on it.                              */
int atlas_debug_tile_wait_hint(unsigned ns);
/* Tuning hook: with on == 0, node-group tables built afterwards keep      */
/* every group in per-node form; 1 (the default) stores the groups whose   */
/* union of stencil rows matches their operator's pattern in union form    */
/* (tiles of one consumer warp per group only; see                          */
/* atlas_fvm_tile_union_groups).  Results do not depend on it.             */
int atlas_debug_tile_unions(int on);
/* Inspection: in *n, how many groups of the node-group tables of op for   */
/* fields of dtype are stored in union form: each distinct neighbour row   */
/* of the group's four nodes read once and applied to every node whose     */
/* stencil row holds it, in that row's order (the sums are those of the    */
/* per-node form, operation for operation).  Builds the tables with the    */
/* operator's current launch shape; 0 when there are none (F64, or tiles   */
/* of two warps per group).                                                 */
int atlas_fvm_tile_union_groups(atlas_fvm_t f, int op, int dtype, int64_t* n);
/* Inspection: copy out the FP64 node-group table of one operator: the    */
/* union of each group's stencil rows (the node-group kernels' tiles are   */
/* cut from these groups, and stage exactly these neighbours).  Groups     */
/* are runs of up to four consecutive nodes of a grid row.  head[g][4] =   */
/* {first node, first entry, end entry, nb | count << 16 | imask << 20}:   */
/* entries [first entry, end entry) are the distinct neighbours of the     */
/* group's nodes in ascending id order; nb of them come before the run of  */
/* the group's own nodes, whose offsets from the first node imask marks.   */
/* hdr[e] = j | mask << 28: neighbour j and the group's nodes (bit t: node */
/* first + t) whose stencil row holds j.  w[e][t][2] = that node's weights */
/* towards j as in atlas_fvm_stencil_table (0 where the bit is clear).     */
/* Call once with NULL arrays for the counts.  Host only; ATLAS_EINVAL     */
/* when the stencil has no group table (then the per-node kernels run).    */
int atlas_fvm_group_table(atlas_fvm_t f, int op, int64_t* ngroups, int64_t* nent, int32_t* head, uint32_t* hdr,
                          double* w);
/* Inspection: copy out the FP32 tile table of one operator's node-group  */
/* kernels, cut into tiles of groups_per_tile (1..11) groups spanning      */
/* rows_per_tile (1..3) grid rows (see atlas_fvm_set_group), with union    */
/* groups when unions != 0 (as for tiles of one warp per group).           */
/* head[t][72] = {first node, groups, ranges, slots, blob offset (16-byte  */
/* units), blob bytes, 0, 0}, then per copy range {first node, count,      */
/* first slot, 0}; the staged row of slot s is the s-th smallest node id  */
/* of the ranges.  blob: per tile {groups, 0, first node, 0}, per group    */
/* {slot of its first node, word offset of its data, its first node,       */
/* count | regular << 16 | union << 17 | D << 20}, the B term              */
/* [groups][4][2] (operators with one), then each group's data.  Per-node */
/* form: slots [D][4], weights [D][4][nw][2] (each weight twice).  Union   */
/* form (D = U): slots [U] (padded to four words), then per entry and per */
/* node whose stencil row holds it, in node order, its nw weights.        */
/* Units: unit u covers nodes unit_first[u] .. unit_first[u + 1] - 1 with */
/* tiles unit_tile[u] .. unit_tile[u + 1] - 1 (nunits + 1 entries each).  */
/* Call once with NULL arrays for the counts.  Host only; ATLAS_EINVAL     */
/* when the stencil has no tile table.                                     */
int atlas_fvm_tile_table(atlas_fvm_t f, int op, int groups_per_tile, int rows_per_tile, int unions, int64_t* ntiles,
                         int64_t* nwords, int32_t* head, uint32_t* blob, int64_t* nunits, int64_t* unit_first,
                         int32_t* unit_tile);
void atlas_fvm_destroy(atlas_fvm_t f);

/* ---------------------------------------------------------------------- */
/* Nabla operators (paper Sec. 2.3: gradient, divergence, Laplacian).      */
/* Every operator is deterministic: no atomics, fixed summation order.    */
/* ---------------------------------------------------------------------- */
/* Gradient: gx = (1/V_i) sum_e n_ie,lon (f_j - f_i)/2,                    */
/*           gy = (cos(lat_i)/V_i) sum_e n_ie,lat (f_j - f_i)/2,           */
/* summed over the edges e = (i, j) of node i including its pole edge;     */
/* n_ie = +-S_e (sign of i in e) on regular edges and S_e on pole edges.   */
/* Because every dual cell is closed this equals the Green's-theorem form  */
/* with face values (f_a + f_b)/2.  Units: 1/m.  in: f; out: gx, gy.       */
int atlas_nabla_gradient(atlas_fvm_t fvm, const void* f, void* gx, void* gy, int nlev, int64_t ld,
                         atlas_dtype dtype, void* stream);
/* Divergence of the vector (u, v) in physical components:                 */
/* V_i div_i = sum_{regular e} n_ie . (F_j - F_i)/2 - F_i . n_pole,i,      */
/* F = (u, v cos(lat)): the flux form with zero flux through the pole.     */
int atlas_nabla_divergence(atlas_fvm_t fvm, const void* u, const void* v, void* div, int nlev,
                           int64_t ld, atlas_dtype dtype, void* stream);
/* Laplacian = divergence of the gradient, applied as one fused two-ring   */
/* stencil L = D G (no intermediate field).                                */
int atlas_nabla_laplacian(atlas_fvm_t fvm, const void* f, void* lap, int nlev, int64_t ld,
                          atlas_dtype dtype, void* stream);
/* Adjoints: the exact transposes of the gradient (f = G^T (gx, gy)) and   */
/* divergence ((u, v) = D^T d) maps, written as gathers.                   */
int atlas_nabla_gradient_adjoint(atlas_fvm_t fvm, const void* gx, const void* gy, void* f, int nlev,
                                 int64_t ld, atlas_dtype dtype, void* stream);
int atlas_nabla_divergence_adjoint(atlas_fvm_t fvm, const void* div, void* u, void* v, int nlev,
                                   int64_t ld, atlas_dtype dtype, void* stream);
/* Curl (vertical vorticity) of the tangent vector (u, v) in physical      */
/* components, zeta = (1/(R cos lat)) [d_lon v - d_lat (u cos lat)], by    */
/* Stokes' theorem on the dual cell (paper Sec. 2.3 lists curl among the  */
/* operators): V_i zeta_i is the circulation around cell i, the flux of    */
/* G = (v, -u cos(lat)) through its faces with face means, in the         */
/* closure-exact form sum_{regular e} n_ie . (G_j - G_i)/2 - G_i . n_pole */
/* (no circulation on the pole segment).  curl(u, v) = div(v, -u).         */
/* Units: 1/s for u, v in m/s.  in: u, v; out: zeta.                       */
int atlas_nabla_curl(atlas_fvm_t fvm, const void* u, const void* v, void* zeta, int nlev, int64_t ld,
                     atlas_dtype dtype, void* stream);
/* Curl adjoint (u_bar, v_bar) = C^T zeta_bar: the exact transpose of the  */
/* curl as a linear map (column i of C gathered at node i from the rows of */
/* its regular-edge neighbours, as the other adjoints), for variational    */
/* (reverse-mode) use of the curl.  in: zeta; out: u, v (must not overlap  */
/* the input or each other).                                               */
int atlas_nabla_curl_adjoint(atlas_fvm_t fvm, const void* zeta, void* u, void* v, int nlev, int64_t ld,
                             atlas_dtype dtype, void* stream);
/* Gradient of both physical components of a tangent vector field:         */
/* (ux, uy) = grad u, (vx, vy) = grad v, as atlas_nabla_gradient except on */
/* the pole edge: a polar node and its antipode (its pole-edge neighbour)  */
/* have opposite local east and north directions, so the antipode's        */
/* component enters the pole-face mean with its sign reversed (face value  */
/* (f_i - f_j)/2, closure-exact term -n_pole (f_i + f_j)/2).  Two launches */
/* of the same kernel, one per component.  Outputs must not overlap the   */
/* inputs or each other.                                                   */
int atlas_nabla_vector_gradient(atlas_fvm_t fvm, const void* u, const void* v, void* ux, void* uy, void* vx,
                                void* vy, int nlev, int64_t ld, atlas_dtype dtype, void* stream);

/* ---------------------------------------------------------------------- */
/* Edge-based two-kernel forms of the operators of paper Sec. 2.3 (the    */
/* paper gives no kernel design): an edge-flux kernel writes one flux per  */
/* edge and level into a caller-owned device workspace, then a node-gather */
/* kernel sums each node's CSR row of fluxes.  Same results as the fused   */
/* calls up to rounding.  ws must hold atlas_nabla_workspace_bytes(...)    */
/* bytes, 256-byte aligned; its contents on entry are ignored.             */
/* ---------------------------------------------------------------------- */
size_t atlas_nabla_workspace_bytes(atlas_fvm_t fvm, int op, int nlev, int64_t ld, atlas_dtype dtype);
int atlas_nabla_gradient_edges(atlas_fvm_t fvm, const void* f, void* gx, void* gy, void* ws,
                               size_t ws_bytes, int nlev, int64_t ld, atlas_dtype dtype, void* stream);
/* The gradient of atlas_nabla_gradient_edges with the edge flux in the    */
/* averaged (Green-Gauss) form S_e (f_a + f_b)/2, entering the two ends of  */
/* a regular edge with opposite signs and both ends of a pole edge with +1 */
/* (the same operator up to the cells' closure residual, sum_e n_ie).  A   */
/* selectable variant of the edge-flux kernel for comparison: in FP32 its  */
/* node sums cancel terms of size |f| |S_e| / V_i, about R/h times the     */
/* result (~800 at O1280), so its error is that much larger than the       */
/* difference form's.  Same workspace as atlas_nabla_gradient_edges.       */
int atlas_nabla_gradient_edges_averaged(atlas_fvm_t fvm, const void* f, void* gx, void* gy, void* workspace,
                                        size_t ws_bytes, int nlev, int64_t ld, atlas_dtype dtype, void* stream);
int atlas_nabla_divergence_edges(atlas_fvm_t fvm, const void* u, const void* v, void* div, void* ws,
                                 size_t ws_bytes, int nlev, int64_t ld, atlas_dtype dtype, void* stream);
/* grad into ws, then div of it: the two-pass Laplacian.                   */
int atlas_nabla_laplacian_edges(atlas_fvm_t fvm, const void* f, void* lap, void* ws, size_t ws_bytes,
                                int nlev, int64_t ld, atlas_dtype dtype, void* stream);

/* The two-pass Laplacian without any allocation.  The paper has no        */
/* counterpart; it is for callers that cannot call cudaMalloc when they    */
/* apply the operator: code running inside another framework's memory     */
/* pool or a pre-sized arena, code in a phase that must not allocate or    */
/* synchronise, and callers with no device allocator of their own (a       */
/* Fortran or C model holding only field pointers).  Instead of a caller   */
/* workspace it uses a static device array owned by the library, of 64 MiB */
/* (67108864 bytes), which every GPU that loads the library holds until    */
/* the process exits.  Sizes whose                                         */
/* workspace (atlas_nabla_workspace_bytes with ATLAS_OP_LAPLACIAN) exceeds */
/* it are rejected with ATLAS_EINVAL.  The call builds no tables: prepare  */
/* them first with atlas_fvm_prepare (gradient and divergence bits, this   */
/* dtype), otherwise it returns ATLAS_ESTATE.  The first call on a device, */
/* with that device current, looks up the array's device address once;    */
/* make that first call before any stream capture.  The address stays     */
/* cached for the process: after cudaDeviceReset (which also invalidates   */
/* every fvm's device tables) the entry point must not be called again.    */
/* All calls share the array and it keeps the last call's contents;        */
/* nothing in it needs to start at zero: both passes use one vector width, */
/* so every value the second pass reads, padding lanes included, was       */
/* written by the first pass of the same call.  Calls that overlap on the  */
/* GPU race on it.  F32 or F64 fields.                                     */
int atlas_nabla_laplacian_edges_noalloc(atlas_fvm_t fvm, const void* f, void* lap, int nlev, int64_t ld,
                                        atlas_dtype dtype, void* stream);

/* ---------------------------------------------------------------------- */
/* Batched launch: the gradient and divergence of paper Sec. 2.3 on many  */
/* fields of different grids and level counts in one persistent kernel    */
/* (one launch, capturable in a CUDA graph; optionally the largest fields  */
/* in plain launches of their own).  The paper has no counterpart.         */
/* ---------------------------------------------------------------------- */
typedef struct {
  int op;              /* ATLAS_OP_GRADIENT or ATLAS_OP_DIVERGENCE           */
  atlas_fvm_t fvm;     /* geometry of this field's grid                      */
  const void* in0;     /* f (gradient) or u (divergence)                     */
  const void* in1;     /* NULL (gradient) or v (divergence)                  */
  void* out0;          /* gx (gradient) or div (divergence)                  */
  void* out1;          /* gy (gradient) or NULL                              */
  int nlev;
  int64_t ld;
} atlas_batch_desc;
/* Work split: each descriptor is cut into tiles of tile_items (node,      */
/* level-vector) items (default 1024), each computed by one block; vec    */
/* levels per thread (1, 2 or 4; the batch uses the widest vec that every */
/* field's ld and pointers allow, capped by this value), threads per       */
/* block (64..256, default 256), blocks per SM of the persistent grid      */
/* (0 = as many as fit), and plain_waves: fields of at least plain_waves  */
/* full GPU waves (plain_waves x 2048 x SMs items) run as plain launches  */
/* with their operator's own kernel and launch shape inside               */
/* atlas_batch_launch, the others in the persistent launch (0: the        */
/* default, 4 waves; -1: every field in the persistent launch).  Zero     */
/* fields take the defaults.                                               */
typedef struct {
  int vec;
  int tile_items;
  int threads;
  int blocks_per_sm;
  int plain_waves;
} atlas_batch_tune;
/* n = 1..256 descriptors (split larger sets into several batches).       */
/* Validates the descriptors and prepares every fvm's tables.  The         */
/* descriptor table is kept by the batch and passed whole to every launch  */
/* as a kernel parameter (no device allocation).  dtype is ATLAS_F32 or    */
/* ATLAS_F64 for all fields of the batch.  The field pointers are fixed at */
/* creation; re-create the batch for other fields.                         */
int atlas_batch_create(const atlas_batch_desc* descs, int n, atlas_dtype dtype, const atlas_batch_tune* tune,
                       atlas_batch_t* out);
/* One persistent launch over the tiles of every field (with plain_waves  */
/* set, the fields that large first get plain launches of their own):     */
/* block b computes tiles b, b + grid, ... (divergence tiles, and fields   */
/* with more levels, first).  Results                                      */
/* are bitwise those of plain launches and do not depend on the tile order */
/* or the launch shape (each item is computed once, in CSR order).  A      */
/* launch reads only                                                       */
/* its kernel parameters and the fields, so launches of one batch may be   */
/* captured in CUDA graphs and replayed on any stream.                     */
int atlas_batch_launch(atlas_batch_t b, void* stream);
/* Total tiles and total (node, level) pairs of the batch.                  */
int atlas_batch_info(atlas_batch_t b, int64_t* tiles, int64_t* node_levels);
void atlas_batch_destroy(atlas_batch_t b);

/* ---------------------------------------------------------------------- */
/* Remapping between grids (paper Sec. 4.3, Fig. 6: a field on an O32 grid */
/* remapped to an F8 grid by a linear element-based interpolation in 3D on */
/* the sphere).  Every target point (unit vector p) is located in the      */
/* source mesh triangle whose plane the ray from the centre along p        */
/* crosses inside the triangle; its three weights are the barycentric      */
/* coordinates of that crossing (of several containing triangles: the one  */
/* whose smallest weight is largest, then the lowest triangle id).  Built  */
/* on the host; fails with ATLAS_EINVAL if a target lies in a polar cap    */
/* (north of the source's first row or south of its last), which no        */
/* triangle covers.  The source must be a global mesh (O<N> or F<N>); any */
/* grid, a regional one included, can be the target.  The remap keeps its */
/* mesh and grid alive.                                                    */
/* ---------------------------------------------------------------------- */
int atlas_remap_create(atlas_mesh_t src, atlas_grid_t dst, atlas_remap_t* out);
/* Views valid until atlas_remap_destroy: ntgt (the target grid's points), */
/* nodes[ntgt][3] source node ids and weights[ntgt][3].                    */
int atlas_remap_info(atlas_remap_t r, int64_t* ntgt, const int32_t** nodes, const double** weights);
/* dst[t][k] = sum_q weights[t][q] src[nodes[t][q]][k] for the targets t    */
/* and levels k < nlev: src is a field[source node][ld_src], dst a          */
/* field[target][ld_dst] (device pointers, one dtype).  Padding levels of  */
/* dst up to the end of the last 16-byte vector are set to zero when       */
/* ld_dst allows whole vectors.  Tables are uploaded on the first call of   */
/* a precision.                                                            */
int atlas_remap_apply(atlas_remap_t r, const void* src, void* dst, int nlev, int64_t ld_src, int64_t ld_dst,
                      atlas_dtype dtype, void* stream);
void atlas_remap_destroy(atlas_remap_t r);

/* ---------------------------------------------------------------------- */
/* Band partitions (paper Sec. 2.3: a mesh may be split into partitions,  */
/* one per MPI task, with overlap regions filled by halo exchange).        */
/* nparts parts split the rows north to south into                         */
/* consecutive bands of about equal node counts; part p owns the node      */
/* range [own0, own1) (whole rows) and reads the halo range               */
/* [halo0, halo1) = its rows plus halo_rings (1 or 2) rows on each side,   */
/* which is every value its nodes' stencils touch (two rings: the fused    */
/* Laplacian).  Each part has at least halo_rings rows, so a halo row      */
/* belongs to the adjacent part: one exchange per side refreshes it.       */
/* Host only (works without a GPU).                                        */
/* ---------------------------------------------------------------------- */
typedef struct atlas_part_s* atlas_part_t;
int atlas_part_create(atlas_fvm_t f, int nparts, int part, int halo_rings, atlas_part_t* out);
int atlas_part_info(atlas_part_t p, int64_t* own0, int64_t* own1, int64_t* halo0, int64_t* halo1);
/* Exchange with the part before (side 0, north) or after (side 1, south): */
/* peer = that part's index or -1; this part sends its own nodes           */
/* [send0, send1) and receives [recv0, recv1) into its halo.  The peer's   */
/* recv range is this part's send range and the other way round.           */
int atlas_part_neighbour(atlas_part_t p, int side, int* peer, int64_t* send0, int64_t* send1, int64_t* recv0,
                         int64_t* recv1);
/* Apply operator op (ATLAS_OP_*) to this part's own nodes.  Inputs are    */
/* local fields of halo1 - halo0 rows (row k = node halo0 + k, halo rows   */
/* filled by the exchange), outputs local fields of own1 - own0 rows (row */
/* k = node own0 + k); ld, dtype and stream as for the whole-grid calls.   */
/* Results equal the whole-grid operator's on these nodes, bitwise (same   */
/* kernels and summation order).  For ATLAS_OP_VECTOR_GRADIENT the call    */
/* takes one component (in0) and writes its two gradient components.      */
/* The Laplacian needs halo_rings = 2.                                     */
int atlas_part_apply(atlas_part_t p, int op, const void* in0, const void* in1, void* out0, void* out1, int nlev,
                     int64_t ld, atlas_dtype dtype, void* stream);
/* Overlap of the halo exchange with computation (the asynchronous        */
/* communication the paper aims for, Sec. 2.2.3): the interior range       */
/* [inner0, inner1) holds the own nodes whose stencils read no halo row    */
/* (own rows at least halo_rings rows from each side that has a            */
/* neighbour), computable while the exchange is in flight; the own nodes   */
/* outside it need the exchanged halo.  inner0 == inner1 when a part has   */
/* no interior.                                                            */
int atlas_part_interior(atlas_part_t p, int64_t* inner0, int64_t* inner1);
/* atlas_part_apply restricted to own nodes [node0, node0 + count) within  */
/* [own0, own1): inputs as for atlas_part_apply (halo-range fields), the   */
/* outputs still own-range fields (row k = node own0 + k; only rows of the */
/* range are written).  Same results, bitwise, as the whole own range.     */
int atlas_part_apply_nodes(atlas_part_t p, int op, const void* in0, const void* in1, void* out0, void* out1,
                           int64_t node0, int64_t count, int nlev, int64_t ld, atlas_dtype dtype, void* stream);
void atlas_part_destroy(atlas_part_t p);

/* ---------------------------------------------------------------------- */
/* Field synchronisation (paper Sec. 4.2: update_host after device work).  */
/* One cudaMemcpyAsync of bytes from src to dst on stream; direction 0 =   */
/* host to device, 1 = device to host, 2 = device to device.  Host memory  */
/* should be pinned for the copy to be asynchronous.                       */
/* ---------------------------------------------------------------------- */
int atlas_field_sync(void* dst, const void* src, size_t bytes, int direction, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ATLAS_GB_H */
