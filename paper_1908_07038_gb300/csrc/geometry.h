// Host-side grid, mesh and median-dual geometry of the octahedral reduced
// Gaussian grid, plus the per-operator stencil tables the GPU kernels read.
//
// The paper's workflow is Grid -> Mesh -> FunctionSpace -> Field, with
// gradient, divergence and Laplacian supplied on top (Sec. 2.3, Fig. 2).  This
// file builds the Grid (Gaussian latitudes, octahedral rows), the Mesh (zipper
// triangulation, pole edges, node->edge CSR) and the FunctionSpace geometry
// (median-dual volumes and normals, FP64), all on the host.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace atlasgb {

struct Grid {
  int N = 0;
  int nlat = 0;
  bool octahedral = true;      // false: regular (full) Gaussian grid F<N>
  int64_t nnodes = 0;
  std::vector<int32_t> pl;     // points per row, north -> south
  std::vector<int64_t> off;    // first node of each row, size nlat+1
  std::vector<double> colat;   // colatitude of each row (radians)
  std::vector<double> lat;     // latitude of each row (radians)
  std::vector<double> lonlat;  // [nnodes][2] longitude, latitude (radians)
  // regional (limited-area) grids: projection >= 0, nlat rows of nx points
  int projection = -1;         // -1: global; else a RegionalProjection
  int nx = 0;
  double proj_params[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<double> xy;      // [nnodes][2] plane coordinates on the unit sphere
  std::vector<double> h;       // [nnodes][2] scale factors h_x, h_y on the unit sphere
  bool regional() const { return projection >= 0; }
};

struct Mesh {
  const Grid* grid = nullptr;
  int64_t nedges = 0, ntri = 0;
  std::vector<int32_t> e2n;       // [E][2], a < b, sorted by (a, b)
  std::vector<uint8_t> is_pole;   // [E]
  std::vector<int32_t> n2e_ptr;   // [V+1]
  std::vector<int32_t> n2e;       // [2E], ascending edge id per node
  std::vector<int8_t> n2e_sign;   // [2E], +1 at a, -1 at b
  std::vector<int32_t> tri;       // [T][3] node ids, band by band
  // dual-face end points of every regular edge: side 0 = left of a->b, 1 = right
  std::vector<double> side_off;   // [E][2] offset of the end point from the edge midpoint (turns)
  std::vector<double> side_lat;   // [E][2] latitude of the end point
  std::vector<double> mid_lat;    // [E]
};

struct Dual {
  double R = 0;
  std::vector<double> S;          // [E][2] (S_lambda, S_phi) oriented a -> b
  std::vector<double> V;          // [V]
  std::vector<double> coslat;     // [V]
  std::vector<double> pole_nphi;  // [V] phi-normal of the pole segment (0 off the polar rows)
  // regional grids only: S holds R times the plane normals of the dual faces
  std::vector<double> A;          // [V] R^2 times the plane area of the dual cell
  std::vector<double> Sb;         // [E][2] R times the outward plane normal of a boundary edge, else 0
};

// A node-centred stencil: out_c(i) = sum_{q in row i} sum_m W_{c,m}(q) (x_m(nbr[q]) - x_m(i))
//                                    + sum_m B_{c,m}(i) x_m(i)
// with one (NIN = 1) or two (NIN = 2) inputs and one or two outputs.  The
// weight pair w[2q], w[2q+1] is (W_{0,0}, W_{1,0}) when NIN = 1 and
// (W_{0,0}, W_{0,1}) when NIN = 2; b[2i], b[2i+1] likewise.  Entry order in
// a row (build_stencil): the neighbours on the node's own grid row at
// offsets -2, -1, +1, +2 along the row (those present), then the others by
// ascending id; every kernel sums a node's terms in this order.
struct Stencil {
  int nin = 1, nout = 1;
  bool has_b = false;
  bool scalar_w = false;          // only w[2q] is used (Laplacian)
  std::vector<int32_t> ptr;       // [V+1]
  std::vector<int32_t> nbr;       // [nnz]
  std::vector<double> w;          // [nnz][2]
  std::vector<double> b;          // [V][2] (empty when !has_b)
};

// Edge-based two-pass data (edge-flux kernel + node-gather kernel).
struct EdgeGather {
  std::vector<int32_t> ptr;       // [V+1]
  std::vector<int32_t> ent;       // [nnz] edge id << 1 | (negative sign)
  std::vector<double> inv_v;      // [V] 1/V
  std::vector<double> cos_v;      // [V] cos/V
  std::vector<double> pole_coef;  // [V] -cos * n_pole / V (divergence), 0 off the polar rows
  std::vector<double> dcos;       // [E] cos(b) - cos(a)
};

void gauss_colatitudes(int n, double* theta);
bool build_grid(int N, Grid& g);
bool build_mesh(const Grid& g, Mesh& m);
bool build_dual(const Mesh& m, double R, Dual& d);

enum StencilOp {
  OP_GRAD = 0,
  OP_DIV = 1,
  OP_GRAD_ADJ = 2,
  OP_DIV_ADJ = 3,
  OP_LAP = 4,
  OP_CURL = 5,   // vertical vorticity of (u, v): two inputs, one output
  OP_VGRAD = 6,  // gradient of one component of a tangent vector field
  OP_CURL_ADJ = 7,  // adjoint of the curl: one input, two outputs
  OP_COUNT = 8
};
bool build_stencil(const Mesh& m, const Dual& d, int op, Stencil& s);
// averaged: the gradient's edge flux in the averaged form S_e (x_a + x_b)/2
// (enters a with +1, b with -1 on regular edges, both ends with +1 on pole
// edges) instead of the difference form S_e (x_b - x_a)/2.
bool build_edge_gather(const Mesh& m, const Dual& d, int op /*OP_GRAD or OP_DIV*/, EdgeGather& eg,
                       bool averaged = false);

// Node-group table of a stencil (the warp-per-group kernels).  Each row of
// the grid is cut into groups of up to kGroup consecutive nodes; a group's
// table is the union of its nodes' stencil rows, sorted by neighbour id, one
// entry per distinct neighbour j with a mask of the group's nodes whose row
// holds j and, for each node of the group, its weight(s) towards j (0 where
// the mask bit is clear).  Every node therefore meets its own terms in the
// order of its per-node row, so applying the group table gives the same sums
// as the per-node table, operation for operation.  The group's own nodes
// that appear as neighbours form one contiguous run of the sorted entries
// (ids first .. first + count - 1); the kernels take their values from the
// registers that already hold them.
constexpr int kGroup = 4;
struct GroupStencil {
  int nw = 1;                   // weights per (entry, node): 1 (scalar weights) or 2
  // [ng][4]: first node, first entry q0, end entry q1,
  //          nb | count << 16 | imask << 20, where nb entries precede the
  //          internal run and imask marks the group's nodes that occur in it
  std::vector<int32_t> head;
  std::vector<uint32_t> hdr;    // [nent]: j | mask << 28 (j < 2^28)
  std::vector<double> w;        // [nent][kGroup][nw]
  std::vector<int64_t> first;   // [ng + 1]: first node of every group, then nnodes
  std::vector<uint8_t> row_start;  // [ng]: 1 where the group begins a grid row
};
// Fails (false) when a per-node row is not strictly ascending, a node id
// does not fit in 28 bits or the entry count overflows 32 bits; the caller
// then keeps the per-node kernels.
bool build_group_stencil(const Stencil& s, const Grid& g, GroupStencil& gs);

// Tile table of the shared-memory node-group kernels, built from a group
// table.  Tiles hold groups of one to three consecutive grid rows (see
// build_tile_stencil).  A tile lists the node rows its groups read (their own
// nodes and all their neighbours) as at most kTileRanges runs of
// consecutive node ids; the kernel copies those runs into shared memory in
// order, so the node with the s-th smallest id of the list sits in slot s.
//   head[t][kTileHead]: first node, groups, ranges, slots (rows staged),
//     blob offset (16-byte units), blob bytes, 0, 0, then per range
//     (first node, count, first slot, 0).
//   blob: per tile, 16-byte aligned: {groups, 0, first node, 0}; per group
//     {slot of its first node, word offset of its data in the blob, its
//     first node, count | regular << 16 | union << 17 | D << 20}
//     (regular: four nodes whose first R entries, R
//     = 2 for one-ring tables and 4 for the Laplacian, are their row
//     neighbours at offsets -1, +1, resp. -2, -1, +1, +2 wherever that
//     neighbour belongs to the group, and D >= R); the B term
//     [groups * 4][2] (floats; operators with one); then
//     per group, D being its nodes' longest stencil row: slots [D][4]
//     (entry e of node t: its row's e-th neighbour, or its own slot past its
//     row's end) and weights [D][4][nw] as f32x2 pairs (each weight twice;
//     0 past the row's end).
// With unions, a group of four nodes whose union of rows matches its
// operator's pattern (patterns.h) is stored in union form instead: its
// header's word 3 has bit 17 set and D (bits 20..27) = U, and its data are the slots of
// the U union entries (padded to a multiple of four words), then, entry by
// entry and for each node holding the entry in node order, its nw weights
// as floats (padded likewise).  Only kernels that give each group one warp
// read union groups.
constexpr int kTileRanges = 16;
constexpr int kTileHead = 8 + 4 * kTileRanges;
constexpr int kMaxTileRows = 3;   // grid rows a tile may span
constexpr int kMaxTileRow = 255;  // longest stencil row a per-node group may have (8 bits of its header)
struct TileStencil {
  int nw = 1;
  int groups_per_tile = 7;
  int rows_per_tile = 1;
  bool unions = false;
  int64_t union_groups = 0;       // groups stored in union form
  int64_t ntiles = 0;
  std::vector<int32_t> head;      // [ntiles][kTileHead]
  std::vector<uint32_t> blob;     // 32-bit words
  // units: runs of whole grid rows whose tiles are consecutive; unit u
  // holds nodes first[u] .. first[u + 1] - 1 and tiles unit_tile[u] ..
  // unit_tile[u + 1] - 1 (a launch covers whole units)
  std::vector<int64_t> first;     // [nunits + 1], then nnodes
  std::vector<int32_t> unit_tile; // [nunits + 1], then ntiles
  int32_t max_slots = 0;          // most rows any tile stages
  int32_t max_blob = 0;           // largest tile blob (bytes)
  int32_t max_groups = 0;         // most groups any tile holds
};
// Tiles span rows_per_tile (1..kMaxTileRows) consecutive grid rows, with up
// to groups_per_tile / rows_per_tile groups of each; a unit of rows one of
// whose tiles would need more than kTileRanges copy runs is tiled row by
// row instead.  Fails (false) when a single-row tile needs more than
// kTileRanges runs or a stencil row is longer than kMaxTileRow (the caller
// keeps the per-node kernels).
bool build_tile_stencil(const GroupStencil& gs, const Stencil& s, int groups_per_tile, TileStencil& ts,
                        bool unions = false, int rows_per_tile = 1);

// Regular (full) Gaussian grid F<N>: the 2N Gaussian latitudes of O<N>, each
// with 4N longitudes j/(4N) turns.  A remapping target, and meshed by the
// same zipper as O<N>.
bool build_regular_gaussian_grid(int N, Grid& g);

// Remapping weights (remap.cpp): for every target (lon, lat) in radians, the
// three source nodes nodes[3t..3t+2] and weights of the linear interpolation
// in three-dimensional space over the sphere in the source mesh's triangle
// that contains it.
// not_located counts targets in no triangle (the polar caps); their nodes
// are -1 and weights 0.  Returns false on an inconsistent mesh.
bool build_remap(const Mesh& m, const double* tgt_lonlat, int64_t ntgt, std::vector<int32_t>& nodes,
                 std::vector<double>& weights, int64_t& not_located);

// Regional (limited-area) grids (regional.cpp): a rectangle of a map
// projection, nx points per row and ny rows, triangulated two triangles per
// quad, with the median dual built in the projection plane.  The operators
// follow the orthogonal-coordinate forms with the projection's scale factors
// h_x, h_y taken at the nodes, and give vector components along the grid's
// x and y directions.
enum RegionalProjection {
  PROJ_ROTATED_LONLAT = 0,  // x, y = rotated longitude, latitude (degrees)
  PROJ_MERCATOR = 1,        // x, y in metres on a sphere of radius p[4]
  PROJ_LAMBERT_CONFORMAL = 2,  // tangent cone, x, y in metres
  PROJ_POLAR_STEREOGRAPHIC = 3  // tangent at a pole, x, y in metres
};
// params: {xmin, xmax, ymin, ymax, p4, p5, p6, p7} as documented in atlas_gb.h.
// Returns false with a reason in why on an invalid domain.
bool build_regional_grid(int projection, int nx, int ny, const double* params, Grid& g, const char** why);
bool build_regional_mesh(const Grid& g, Mesh& m);
bool build_regional_dual(const Mesh& m, double R, Dual& d);
bool build_regional_stencil(const Mesh& m, const Dual& d, int op, Stencil& s);
// Consistency of a mesh and its dual (any grid): the node->edge CSR covers
// every edge exactly twice, at its first node with sign +1 and at its second
// with -1; edge ends are in range with a < b; and every dual cell closes: the
// sum of its outward face normals (pole faces counted at both ends; half of
// each boundary edge's normal on regional grids) is at most tol times the sum
// of their absolute values.  On failure returns false with the first bad
// node (or -1) and a reason; worst is the largest relative closure residual.
bool check_geometry(const Mesh& m, const Dual& d, double tol, double& worst, int64_t& bad_node, const char** why);

// Geometry cache (geomio.cpp): the grid, mesh and dual written to a file and
// read back bit for bit (with a checksum).  load_geometry points m.grid at g;
// its caller then runs check_geometry.
bool save_geometry(const Grid& g, const Mesh& m, const Dual& d, const char* path, const char** why);
bool load_geometry(const char* path, Grid& g, Mesh& m, Dual& d, const char** why);

// Generic table algebra for difference-form stencils with symmetric 1-ring
// sparsity: the transpose (an adjoint) and the product L = D G of a
// two-input divergence-like table with a one-input, two-output
// gradient-like table (the Laplacian; stored without its diagonal, which
// requires G applied to a constant to vanish).
bool transpose_stencil(const Stencil& a, Stencil& t);
bool compose_stencil(const Stencil& d, const Stencil& g, Stencil& l);

}  // namespace atlasgb
