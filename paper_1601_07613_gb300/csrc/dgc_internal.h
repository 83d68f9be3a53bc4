// Internal declarations shared by the host mesh code, the kernels and the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "dgc.h"

namespace dgc {

constexpr int kMaxColors = 15;

// Reference-element tables for one (dim, p).  Volume points carry weights that
// sum to |reference element|; face weights sum to 1 over a face.
struct RefTables {
  int dim = 0, p = 0, np = 0, nqv = 0, nqf = 0, nfaces = 0;
  bool quad = false;  // the square [0,1]^2 with the tensor Legendre space Q_p
  std::vector<double> vr, vs, vt, vw;  // volume points (reference coordinates) and weights
  std::vector<double> phiV;            // [nqv][np]
  std::vector<double> dphiV;           // [dim][nqv][np]
  std::vector<double> fw;              // [nqf] face weights
  std::vector<double> ft;              // 2D: [nqf] edge points' parameters in [0, 1] from the edge's first vertex
  std::vector<double> phiF;            // [nfaces][nqf][np], face points in face parameters
  // triangles: phi_j on half h of local edge f, at edge parameter (h + t_q) / 2,
  // [nfaces][2][nqf][np] (the coarse side of a hanging edge, Sec. 3.2)
  std::vector<double> phiH;
  // quadrilaterals: the normalised 1-D Legendre polynomials l_k(x) =
  // sqrt(2k+1) P_k(2x-1) (phi_{a(p+1)+b}(r, s) = l_a(r) l_b(s)) at the edge
  // points, [nqf][p+1], and at the ends x = 0 and x = 1, [p+1] each
  std::vector<double> eleg, lend0, lend1;
  // quadrilaterals: the 1-D factors of the volume rule (the square's (p+1)^2
  // points are (x_i, x_k)): l_a(x_i) and l_a'(x_i), [p+1][p+1], and weights
  // summing to 1, [p+1]
  std::vector<double> vleg, vdleg, vw1;
  // triangles: phi_j at the vertices (0,0), (1,0), (0,1), [3][np] (the limiter)
  std::vector<double> phiX;
};

// Builds the tables (quadrature + orthonormal basis) for triangles (dim 2),
// quadrilaterals (dim 2, quad) or tetrahedra (dim 3).  Throws
// std::runtime_error on unsupported sizes.
RefTables make_tables(int dim, int p, bool quad = false);

// Tetrahedra: phi_j at the face points of local face f seen through vertex
// permutation o (0..5, kFacePerms) of the face's three vertices:
// out[((f * 6 + o) * nqf + q) * np + j].  o = 0 is the face's own parameterisation.
std::vector<double> tet_face_orient_tables(const RefTables& T);
extern const int kFacePerms[6][3];

// Evaluates the orthonormal basis and its reference gradient at one point.
void basis_eval(int dim, int p, const double* x, double* phi, double* grad /*[dim][np] or null*/,
                bool quad = false);

// Gauss-Jacobi rule with weight (1-x)^alpha on [-1, 1].
void gauss_jacobi(int n, double alpha, double* x, double* w);

struct DeviceMesh;  // defined in the CUDA translation unit

struct Mesh {
  int dim = 0, p = 0, np = 0, M = 0, nfpe = 0, nvpe = 0;
  // quadrilateral (or hybrid triangle/quadrilateral) mesh: nvpe = nfpe = 4, a
  // triangle lists -1 as its fourth vertex and has no face 3 (face_of = -1);
  // nonaffine counts the elements the kernels do not take (quadrilaterals that
  // are not parallelograms, triangles of hybrid meshes): colored only
  bool quad = false;
  int64_t nonaffine = 0;
  // hybrid triangle/quadrilateral mesh (quad with some triangles): each element
  // carries the space of its kind, P_p (tab_tri) or Q_p (tab); states keep
  // (p+1)^2 coefficients per variable, a triangle using the first (p+1)(p+2)/2
  bool hybrid = false;
  // general quadrilaterals (not parallelograms) map the square bilinearly: per
  // element 1 for such an element (original order); they also run on the
  // table-driven kernels (hybrid = true), with their own mass matrices
  std::vector<uint8_t> bil;
  int64_t nv = 0, ne = 0, ns = 0;
  bool periodic = false;
  double L[3] = {0, 0, 0};
  std::vector<double> X;     // [ne][nvpe][dim] unwrapped vertex coordinates
  std::vector<int32_t> ev;   // [ne][nvpe]
  // edge (face) table, original order
  std::vector<int32_t> sl, sr;
  std::vector<int8_t> sql, sqr;
  std::vector<int32_t> face_of;  // [ne][nfpe] -> side (the first of two on a split edge)
  // nonconforming meshes (Sec. 3.2): half (0 or 1) of the right element's local
  // edge that side s covers, -1 for a conforming side; empty when conforming
  std::vector<int8_t> shalf;
  // refinement level of each element (original order; empty: every element 0)
  std::vector<int8_t> level;
  bool refined = false;
  // the mesh before the last dgc_refine, kept for coarsening (a mesh refined
  // again keeps the earlier ones in base_stack)
  struct Base {
    int64_t nv = 0, ne = 0, ns = 0;
    std::vector<double> X;
    std::vector<int32_t> ev, sl, sr, face_of;
    std::vector<int8_t> sql, sqr, color, shalf, level;
    std::vector<uint8_t> flag;  // refined elements
    std::vector<int32_t> elem_new_of_old;  // the coarse mesh's internal element order
    int ncolors = 0;
    // per refined side (original order), where the Sec. 3.2 map takes its color
    // from: rule & 15 = 0: base side src keeps its color, 1 / 2: first / second
    // half of base side src (c, c + K), 3 + k: interior edge of refined base
    // element src parallel to its edge k; rule >> 4 = the level L of the base
    // elements, K = 3 * 2^L
    std::vector<int32_t> color_src;
    std::vector<int8_t> color_rule;
  } base;
  std::vector<Base> base_stack;
  // geometry, original order
  std::vector<double> detJ, Jinv, inradius;  // Jinv [ne][dim][dim] (row k = grad r_k)
  std::vector<double> snormal, smeas;        // [ns][dim] outward normal of the left element, |face|
  RefTables tab;
  RefTables tab_tri;  // hybrid meshes: the triangles' tables (same point counts as tab)
  // coloring and ordering
  int ncolors = 0;
  bool perfect = false;  // every element has exactly one face of each color
  std::vector<int8_t> color;  // original order
  std::vector<int32_t> elem_new_of_old, side_new_of_old, side_old_of_new, color_off;
  // with the color-1 renumbering: elements [0, reached) are those color 1
  // reaches (each exactly once); -1 without the renumbering
  int64_t reached = -1;
  // options
  bool fuse = true;
  int edges_per_block = 64;  // surface-kernel tile of the kernels without a per-class tile
  // triangle RK steps: tile of the first, middle and last colors' FP32 kernels
  // (edges per block, threads per edge 2 or 4); dgc_set_tile, dgc_autotune
  int tile_epb[3] = {64, 64, 64};
  int tile_tpe[3] = {2, 2, 2};
  bool profile = false;
  bool pdl = true;  // programmatic dependent launch of the RK step's kernels
  bool coop = false;  // dgc_rhs of triangle meshes as one cooperative launch
  bool persistent = false;  // triangle surface kernels: one wave of blocks, grid-stride over the color
  // boundary conditions (dgc_set_boundary; triangle meshes, FP64): per side in
  // original order its kind (DGC_BC_*) and state index, the states [n][4], the
  // moving shock x_s = shock[0] + shock[1] y + shock[2] t between the states
  // shock_st[0] (behind) and shock_st[1] (ahead); has_bc: any kind but
  // transmissive; time: the time the boundary states are taken at (the device
  // copy advances with the RK steps and is read back by dgc_get_time)
  std::vector<int8_t> bc_kind, bc_sidx;
  std::vector<double> bc_states;
  double shock[3] = {0.0, 0.0, 0.0};
  int shock_st[2] = {0, 0};
  bool has_bc = false;
  double time = 0.0;
  bool limit = false;  // the limiter after every RK stage (DGC_OPT_LIMITER)
  bool want_enb = false;  // the device keeps the limiter's face neighbours (set by its first use)
  void* prof = nullptr;  // event records (capi.cu)
  // device side
  DeviceMesh* dev = nullptr;
  bool dirty = true;  // host ordering changed since the last upload
  int64_t last_launches = 0;
};

// Host algorithms (mesh.cpp).  They throw dgc::Error on failure.
struct Error {
  dgc_status code;
  std::string msg;
};

Mesh* build_mesh(int dim, int p, int64_t nv, const double* xyz, int64_t ne, const int32_t* ev,
                 const double* periodic_len, bool quad = false);
struct ColorStats {
  int64_t greedy_conflicts = 0, swaps = 0, breaks = 0, deferrals = 0;
};
ColorStats color_faces(Mesh& m, uint64_t seed, int64_t max_swaps);
int color_faces_naive(Mesh& m);
void reorder(Mesh& m, bool renumber, bool reorder_left);
void refine(Mesh& m, const std::vector<uint8_t>& flag);
void coarsen(Mesh& m);
void vol_points(const Mesh& m, double* xyz);
// general quadrilaterals: the bilinear map (point x and Jacobian J[a*2+k] at
// (r, s) of the square) and the inverse mass matrix of element e (np x np)
void bilinear_map(const double* X, double r, double s, double* x, double* J);
std::vector<double> bilinear_mass_inverse(const Mesh& m, int64_t e);
void project(const Mesh& m, const double* vals, double* c);

// Device side (capi.cu).
void device_free(Mesh& m);

}  // namespace dgc
