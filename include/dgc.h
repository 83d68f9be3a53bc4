/*
 * dgc.h -- C ABI of the colored, race-free DG right-hand-side library for GB300.
 *
 * The library evaluates the right-hand side of the modal discontinuous Galerkin
 * discretisation of the Euler equations (Eq. 2 of Giuliani & Krivodonova, "Edge
 * coloring in unstructured CFD codes") on unstructured triangle and tetrahedral
 * meshes, and on quadrilateral and hybrid triangle/quadrilateral meshes
 * (dgc_mesh_create_elem).  The
 * surface integral is evaluated color by color (Algorithm 1): the
 * edges (faces) are colored so that no element has two edges of one color
 * (Sec. 3.1), so all edges of one color scatter their flux projection into both
 * neighbours with plain stores, no atomics and no per-edge buffer.  Elements and
 * edges are renumbered color-major (Sec. 5, Tables 5 and 6).
 *
 * Conventions
 *   - Every call returns a dgc_status; no exception crosses the ABI.  On error
 *     dgc_last_error() returns a thread-local message.  Arguments are validated
 *     before any device work is enqueued.
 *   - Host arrays are plain C arrays in the caller's (original) element and
 *     vertex order.  Device arrays are raw device pointers (e.g. torch tensor
 *     data pointers) in the library's internal (renumbered) element order and
 *     are owned by the caller.  The mesh object owns its host data and the
 *     device copies of connectivity, geometry and basis tables.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work is enqueued on it; calls that take device pointers do not
 *     synchronise the host, except the first device call on a mesh, which
 *     uploads the mesh synchronously (make it before any stream capture).
 *   - A state vector c holds, per element e, the modal coefficients
 *     c[e][m][j] for equation m (M = 4 in 2D, 5 in 3D) and mode j (Np modes),
 *     FP64, contiguous ([E][M][Np]).  Coefficients refer to the basis that is
 *     orthonormal on the reference element (mass matrix = detJ I).
 */
#ifndef DGC_H
#define DGC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgc_mesh dgc_mesh;
typedef struct dgc_batch dgc_batch;

typedef enum {
  DGC_OK = 0,
  DGC_ERR_ARG = 1,            /* bad argument, or call out of order */
  DGC_ERR_MESH = 2,           /* non-manifold face, non-positive Jacobian, bad ids */
  DGC_ERR_COLORING_LIMIT = 3, /* conflict resolution exceeded max_swaps (Sec. 3.1 has
                                 no termination proof); retry with another seed */
  DGC_ERR_UNSUPPORTED = 4,    /* element type / order / option not built */
  DGC_ERR_CUDA = 5,           /* a CUDA runtime call failed */
  DGC_ERR_OOM = 6,            /* host or device allocation failed */
  DGC_ERR_NONFINITE = 7       /* non-finite or non-physical state detected */
} dgc_status;

/* Precision forms.  The two FP32 forms evaluate the flux, quadrature and projection of
 * Eq. 2 in FP32 and keep geometry and the CFL reduction in FP64.  In both the
 * SSP-RK3 stages are carried as FP32 increments delta_{s+1} = b_s (delta_s + dt L(u_s)),
 * b = (1, 1/4, 2/3), around the state u0 at the start of the step, and the state is
 * updated once per step, u = u0 + delta_3, at full precision:
 *   DGC_FP32_MIXED: FP64 state [E][M][Np] (one FP64 FMA per value per step);
 *   DGC_FP32_KAHAN: FP32 pair state (hi + lo per value), updated by Kahan's compensated
 *     summation; no FP64 arithmetic but the CFL reduction.  Triangles.  Its device layout
 *     (dgc_state_bytes) is written and read by dgc_import_state_prec / _export_.
 * DGC_FP64 keeps the state, geometry, fluxes, wave speeds, the CFL reduction and the
 * stage update in FP64.  On triangle meshes of order p >= 2 and on tetrahedral meshes its
 * basis contractions (the traces sum_j phi_j c_j and the projections onto the modes) run
 * as FP32 pairs (hi + lo, 2^-48 relative per value) on the FP32 pipe, on the deviations of
 * the fluxes from the flux of the element's mean (F(u) - F(ub) and F* - F(ub).n, whose omitted parts
 * cancel exactly between each element's volume and faces); on the benchmark workloads
 * the right-hand side is within 3e-13 of the exact one (relative L2), closer than a
 * plain FP64 evaluation of Eq. 2.  Triangle meshes of order 1 and quadrilateral and hybrid
 * meshes evaluate Eq. 2 as written in FP64. */
typedef enum {
  DGC_FP64 = 0,        /* FP64 state, fluxes and stage update (contractions: see above) */
  DGC_FP32_MIXED = 1,  /* FP32 flux with an FP64 state */
  DGC_FP32_KAHAN = 2   /* FP32 flux with a compensated FP32 pair state */
} dgc_prec;

/* Options (dgc_set_option). */
typedef enum {
  DGC_OPT_FUSE = 0,            /* 1 (default): the first color also computes the volume
                                  integral, the last color applies the RK stage update
                                  (closed conforming meshes only); 0: separate volume
                                  kernel, every color read-modify-writes rhs (Alg. 1) */
  DGC_OPT_EDGES_PER_BLOCK = 1, /* surface-kernel tile: edges per thread block (16..128, x16) */
  DGC_OPT_THREADS_PER_EDGE = 2, /* FP32 colored kernels of the RK steps on triangle meshes:
                                   2 (default: one lane per edge side) or 4 (two lanes per side,
                                   which split the edge's quadrature points, the volume integral's
                                   points and the modes of the epilogue); threads per edge x edges
                                   per block <= 256.  The FP64 kernels, dgc_rhs and the
                                   comparators use 2.  Results differ by FP32 summation order. */
  DGC_OPT_PROFILE = 3,          /* 1: record a CUDA event pair around every kernel launch, on
                                   the launch stream, for dgc_profile_collect; 0 (default): off */
  DGC_OPT_GRAPH = 4,            /* batches: 1 (default) capture the step in a CUDA graph on the
                                   first call and replay it; 0: launch the kernels directly */
  DGC_OPT_PDL = 5,              /* meshes: 1 (default) launch the surface and CFL kernels of
                                   dgc_rk_step, dgc_rhs and the comparators with programmatic
                                   dependent launch (each kernel's work that does not read its
                                   predecessor's output overlaps the predecessor's end); 0: plain
                                   stream order.  Results are identical. */
  DGC_OPT_COOPERATIVE = 6,      /* triangle meshes: 1 runs dgc_rhs as one cooperative launch, the
                                   phases of Algorithm 1 (first color with the volume integral,
                                   then each further color) separated by grid-wide barriers
                                   instead of kernel boundaries; 0 (default): one launch per
                                   phase.  Results are identical. */
  DGC_OPT_PERSISTENT = 7,       /* triangle meshes: 1 launches each color's surface kernel with at
                                   most one wave of blocks, every warp looping over the color in
                                   steps of the whole grid (no partly filled last wave); 0: one
                                   block per tile of edges.  Default 0; dgc_refine sets 1 (the
                                   refined region's colors fill less than a wave) and dgc_coarsen
                                   back to a conforming mesh 0.  Results are identical. */
  DGC_OPT_LIMITER = 8           /* conforming triangle meshes, FP64: 1 applies the limiter of
                                   dgc_limit after every stage of dgc_rk_step (and of
                                   dgc_rk_step_static); 0 (default): no limiter.  The FP32 forms
                                   refuse a mesh with the limiter on (DGC_ERR_UNSUPPORTED). */
} dgc_option;

/* Boundary kinds of dgc_set_boundary. */
typedef enum {
  DGC_BC_TRANSMISSIVE = 0,  /* U+ = U- (the default of every boundary face) */
  DGC_BC_WALL = 1,          /* slip wall: U+ = U- with the normal momentum reversed */
  DGC_BC_STATE = 2,         /* U+ = a prescribed state */
  DGC_BC_SHOCK = 3          /* a moving planar shock: the state behind it where x < a + b y + c t */
} dgc_bc;

/* Boundary conditions of a conforming triangle mesh (Sec. 5 runs the double Mach
 * reflection problem of its reference [giuliani] for Table 7; the paper states
 * neither its boundary conditions nor its limiter, and this library's are
 * readings: a slip wall, prescribed inflow states and the moving incident shock
 * on the top boundary, the standard setup of that problem).  kind[s] and
 * state_idx[s] are given per side in the original side order of dgc_get_sides;
 * entries of interior sides are ignored.  At a boundary face the numerical flux
 * takes U- from the element and U+ from its kind: DGC_BC_TRANSMISSIVE U+ = U-;
 * DGC_BC_WALL U+ = (rho, m - 2 (m.n) n, E) with n the element's outward unit
 * normal (no mass or energy crosses the face); DGC_BC_STATE U+ =
 * states[state_idx[s]]; DGC_BC_SHOCK U+ = states[shock_states[0]] where
 * x < shock[0] + shock[1] y + shock[2] t at the face's quadrature point x,
 * else states[shock_states[1]], with t the mesh's time (dgc_set_time; each
 * stage of dgc_rk_step takes t, t + dt, t + dt/2 and the step advances it by
 * dt, on the device).  states: nstates (<= 8) conserved states of 4 doubles;
 * shock and shock_states may be NULL when no face is DGC_BC_SHOCK.  Host
 * arrays, copied.  Every precision form honours them in dgc_rhs, dgc_rk_step,
 * dgc_rk_step_static and the comparators (the FP32 forms evaluate U+ in FP64
 * and take it as a deviation from the element's reference state, like U-);
 * cooperative dgc_rhs and batches refuse a mesh with boundary conditions other
 * than transmissive, and so do dgc_refine and quadrilateral, hybrid and
 * tetrahedral meshes (DGC_ERR_UNSUPPORTED).  DGC_ERR_ARG on a bad kind, state
 * index or count. */
dgc_status dgc_set_boundary(dgc_mesh* mesh, const int8_t* kind, const int8_t* state_idx, int nstates,
                            const double* states, const double* shock, const int8_t* shock_states);

/* The mesh's time, which time-dependent boundary states (DGC_BC_SHOCK) are taken
 * at.  dgc_set_time sets it (0 at creation); dgc_get_time reads the device copy
 * back (synchronising with the device; the host value before the first upload). */
dgc_status dgc_set_time(dgc_mesh* mesh, double t);
dgc_status dgc_get_time(dgc_mesh* mesh, double* t);

/* The limiter, once, in place on an FP64 state c_dev of a conforming triangle mesh
 * (reading: the paper takes its limiter from [giuliani]; this is the
 * Barth-Jespersen limiter on the conserved variables): per element and variable,
 * with u_e the element's mean and u_min, u_max the least and greatest of u_e and
 * its face neighbours' means, every mode j >= 1 is multiplied by the largest
 * alpha in [0, 1] that keeps u_e + alpha (u(x_i) - u_e) within [u_min, u_max] at
 * the element's vertices and volume quadrature points.  Means are unchanged.
 * DGC_OPT_LIMITER applies it after every RK stage.  prec must be DGC_FP64. */
dgc_status dgc_limit(dgc_mesh* mesh, dgc_prec prec, double* c_dev, void* stream);

/* Kernel classes reported by dgc_profile_collect. */
typedef enum {
  DGC_K_CFL = 0,      /* CFL reduction (and FP32 copy of the state, mixed precision) */
  DGC_K_VOLUME = 1,   /* volume integral alone (unfused path) */
  DGC_K_FIRST = 2,    /* first color fused with the volume integral */
  DGC_K_COLOR = 3,    /* a color that read-modify-writes rhs */
  DGC_K_LAST = 4,     /* last color fused with the RK stage update */
  DGC_K_STAGE = 5,    /* RK stage update alone (unfused path) */
  DGC_K_ATOMIC = 6,   /* all edges with atomicAdd (comparator) */
  DGC_K_BUFFER = 7,   /* all edges into the per-edge buffer (comparator) */
  DGC_K_GATHER = 8,   /* per-element gather of the buffer (comparator) */
  DGC_K_LIMIT = 9,    /* the limiter after an RK stage (and the step's time advance) */
  DGC_K_NCLASSES = 16
} dgc_kernel_class;

/* Mesh ingest (Sec. 2 connectivity graph; Sec. 5 edge table).
 * dim = 2 (triangles, CCW vertex order) or 3 (tetrahedra, positive volume).
 * p = polynomial order (triangles 1..3, tetrahedra 1..2 in this build).
 * xyz: nv*dim FP64 vertex coordinates, row-major.  ev: ne*(dim+1) int32 vertex ids.
 * periodic_len: NULL, or dim period lengths; periodic meshes identify faces across
 * the period by shared vertex ids and unwrap each element to lie within half a period
 * of its vertex 0.  Edges are numbered in order of first appearance when the elements
 * and their local faces are scanned (local edge q of a triangle is (v_q, v_{q+1});
 * local face q of a tetrahedron is opposite vertex q); an edge's left element is the
 * first to list it, its right the second (-1 on a boundary).
 * Errors: DGC_ERR_ARG (sizes, pointers), DGC_ERR_MESH (face shared by more than two
 * elements, non-positive Jacobian, vertex id out of range), DGC_ERR_UNSUPPORTED. */
dgc_status dgc_mesh_create(int dim, int p, int64_t nv, const double* xyz, int64_t ne,
                           const int32_t* ev, const double* periodic_len, dgc_mesh** out);

/* Element types of dgc_mesh_create_elem. */
typedef enum { DGC_TRI = 0, DGC_QUAD = 1, DGC_TET = 2 } dgc_elem;

/* Mesh ingest by element type.  DGC_TRI and DGC_TET are dgc_mesh_create with dim 2
 * and 3.  DGC_QUAD: quadrilaterals (Sec. 1 lists them among the meshes the method
 * covers; Sec. 3.1 and Table 2 color them with C = {1, 2, 3, 4}).  ev is ne*4 int32,
 * counterclockwise (every corner must turn left); local edge q is (v_q, v_{q+1 mod 4}).
 * A row whose fourth id is -1 is a triangle: a hybrid triangle/quadrilateral mesh,
 * also colored with 4 colors (Table 2's hybrid mesh).  The reference square [0,1]^2
 * with corners (0,0), (1,0), (1,1), (0,1) at v0..v3 carries the tensor-product
 * Legendre space Q_p, phi_{a(p+1)+b}(r, s) = l_a(r) l_b(s), l_k(x) = sqrt(2k+1)
 * P_k(2x-1) (Np = (p+1)^2, orthonormal on the square; p = 1..3).  A mesh whose
 * elements are all parallelograms (v2 = v1 + v3 - v0 to 1e-12 of the element size)
 * maps them affinely and runs in every precision.  A hybrid mesh, or a mesh with
 * general (non-parallelogram) quadrilaterals, runs in DGC_FP64 and DGC_FP32_MIXED
 * (DGC_FP32_KAHAN: DGC_ERR_UNSUPPORTED) through table-driven kernels (the mixed form:
 * FP32 fluxes and projections of the deviations from each element's mean, an FP64
 * state, right-hand side and stage update; its RK step takes the FP64 step's
 * workspace): its states hold (p+1)^2
 * coefficients per variable for every element, a triangle using the first
 * (p+1)(p+2)/2 (its P_p basis as on triangle meshes; the rest are zero on output);
 * a general quadrilateral maps the square bilinearly, its coefficients refer to the
 * same Q_p basis, its mass matrix int phi_i phi_j detJ is no longer detJ I, and the
 * right-hand side is that of Eq. 2 with this mass matrix inverted.  Such meshes
 * cannot be refined (dgc_refine: DGC_ERR_UNSUPPORTED) and take no two-pass
 * comparator.  A closed quadrilateral mesh with an odd number of elements has no 4-coloring (each
 * color would be a perfect matching of the elements); dgc_color_edges then returns
 * DGC_ERR_COLORING_LIMIT.  Errors as dgc_mesh_create, plus DGC_ERR_MESH for a
 * quadrilateral that is not convex and counterclockwise. */
dgc_status dgc_mesh_create_elem(dgc_elem type, int p, int64_t nv, const double* xyz, int64_t ne,
                                const int32_t* ev, const double* periodic_len, dgc_mesh** out);

/* The mesh's element type (dgc_elem) and the number of its elements that are general
 * (non-parallelogram) quadrilaterals, which only the FP64 table-driven kernels take.
 * Either output may be NULL. */
dgc_status dgc_mesh_element(const dgc_mesh* mesh, int32_t* type, int64_t* nonaffine);

/* Edge (face) coloring of Sec. 3.1 -- modified greedy pass with random nonconflicting
 * colors from C = {1..F} (F = 3 triangles, 4 tetrahedra), then conflict resolution by
 * swaps that do not raise the conflict count, with loop breaking -- followed by the
 * reordering of Sec. 5: edges color-major, the k-th color-1 edge's left/right elements
 * renumbered k and N1+k, colors >= 2 sorted by ascending left element.
 * seed: RNG seed (xorshift64; 0 selects a fixed default).  max_swaps <= 0 selects
 * 1000 * number of edges.  n_colors (out, may be NULL): colors used.  per_color (out,
 * may be NULL, length >= 8): edges per color.  Colors and ordering are bit-identical
 * across runs for a given seed.  Errors: DGC_ERR_COLORING_LIMIT (mesh left uncolored),
 * DGC_ERR_ARG.  Host only; device data is (re)uploaded at the next device call. */
dgc_status dgc_color_edges(dgc_mesh* mesh, uint64_t seed, int64_t max_swaps,
                           int32_t* n_colors, int64_t* per_color);

/* Naive greedy coloring of Sec. 1 (first available color; up to 5 colors on triangles,
 * 7 on tetrahedra), for the color-count ablation of Table 7.  renumber / reorder select
 * the Sec. 5 element renumbering and left-ascending edge order (0 = original order
 * within each color).  Same outputs as dgc_color_edges. */
dgc_status dgc_color_edges_naive(dgc_mesh* mesh, int renumber, int reorder,
                                 int32_t* n_colors, int64_t* per_color);

/* Re-applies the ordering of Sec. 5 to the current coloring with each part switched on or
 * off (the ablation of Table 7): renumber = the color-1 element renumbering, reorder_left
 * = ascending left element within colors >= 2 (0: original order within each color; edges
 * stay color-major).  States imported before the call are in the old element order.
 * DGC_ERR_ARG if the mesh is not colored.  Host only. */
dgc_status dgc_reorder(dgc_mesh* mesh, int renumber, int reorder_left);

/* Sizes: info[0] = E, [1] = edges, [2] = Np, [3] = M, [4] = edge (face) quadrature
 * points, [5] = volume quadrature points, [6] = colors (0 before coloring),
 * [7] = dim, [8] = p, [9] = 1 if every element has exactly one edge of each color. */
dgc_status dgc_mesh_info(const dgc_mesh* mesh, int64_t info[10]);

/* Edge table in original order: left, right (-1 boundary), local face index in left
 * and right (-1 boundary).  Each array has one entry per edge. */
dgc_status dgc_get_sides(const dgc_mesh* mesh, int32_t* left, int32_t* right, int8_t* qleft,
                         int8_t* qright);

/* Nonconforming refinement and its 6-color edge map (Sec. 3.2).  Splits each listed
 * triangle (original element ids; duplicates ignored; n = 0 refines nothing) into four by
 * its edge midpoints, one level per call, on a mesh colored by dgc_color_edges with 3
 * colors or refined before (see below for a second level).
 *   Elements: every refined element is replaced in place by its children [v0, m01, m20],
 *     [m01, v1, m12], [m20, m12, v2], [m01, m12, m20] (new midpoint vertices numbered after
 *     the existing ones, one per split edge in edge order); the original element order of
 *     all later calls is this expanded order.
 *   Colors: a split edge of color c gives its half next to the endpoint with the smaller
 *     vertex id color c and the other half c + 3 (the map ((c + 3m - 4) mod 6) + 1 with the
 *     child number m counted from the smaller vertex id, so both neighbours agree); interior
 *     edges take the color of the parallel parent edge; other edges keep theirs.  The result
 *     uses colors 1..6 and no element has two edges of one color.
 *   Edges: the original edges in order (one edge, or its two halves first-child first),
 *     then three interior edges per refined element.  A half whose other neighbour stays
 *     coarse is a hanging edge: left = the fine child, right = the coarse element, whose
 *     basis is evaluated on that half of its edge (dgc_get_hanging).
 * A refined mesh can be refined again (Sec. 3.2 says the map extends to several levels and
 * gives no rule; reading): an element of level L carries colors 1..K, K = 3 * 2^L, and its
 * split edges' halves take c and c + K (the palette doubles again, colors 1..12 at level 2);
 * the listed elements must have no coarser neighbour (adjacent elements differ by at most one
 * level); an element that is the coarse side of hanging halves may be listed: each half then
 * joins the fine neighbour and the child holding it, with its color, and the interior edge
 * parallel to that edge takes the halves' color modulo K.  At most two levels (12 colors).
 * The mesh is then reordered as by dgc_color_edges (Sec. 5; elements no color-1 edge reaches
 * are numbered last, in original order).  Errors: DGC_ERR_UNSUPPORTED (tetrahedra, a third
 * level), DGC_ERR_ARG (not colored with 3 colors nor refined before, id out of range, an
 * element finer than a neighbour).  Host only; states sized for the old mesh are invalid
 * afterwards. */
dgc_status dgc_refine(dgc_mesh* mesh, int64_t n, const int32_t* elems);

/* Undoes the last dgc_refine (Sec. 3.2): the four children of every element it refined merge
 * back into their parent, and each parent edge takes the color of the child edge parallel to
 * it.  That recovers the coloring before that refinement; the call checks it (DGC_ERR_MESH
 * otherwise) and restores the mesh, its coloring and the Sec. 5 ordering (a mesh refined
 * twice comes back to its first refinement, which a second call undoes).  DGC_ERR_ARG if the
 * mesh is not refined.  Host only; states sized for the refined mesh are invalid afterwards. */
dgc_status dgc_coarsen(dgc_mesh* mesh);

/* Dynamic adaptivity on the device, for a mesh refined by dgc_refine (Sec. 3.2), between the
 * mesh and its last refinement:
 *   dgc_prolong_state: the state of the mesh before refinement (device, [E0][M][Np] FP64
 *     in that mesh's internal order, as it was imported before dgc_refine) to the refined
 *     mesh's state (device, internal order): each child takes the L2 projection of its
 *     parent's polynomial (exact: the child's space contains it); unrefined elements are
 *     copied.
 *   dgc_restrict_state: the refined mesh's state to the state of the mesh before
 *     refinement (call it before dgc_coarsen; the result is in the internal order the mesh
 *     has again after dgc_coarsen): each parent takes the L2 projection of its four
 *     children's piecewise polynomial; unrefined elements are copied.  Restriction after
 *     prolongation is the identity; both conserve the integral of the solution.
 *   Triangle meshes, FP64 states, stream-ordered (the first call after a refinement
 *   uploads the mesh, which allocates).  DGC_ERR_ARG if the mesh is not refined.
 *   dgc_refine_colors_device: the Sec. 3.2 color map of the refined sides evaluated on the
 *     device, one thread per side, from the coloring before refinement (a split edge's
 *     halves take c and c + K, K = 3 * 2^L at the level L of its elements, an interior edge
 *     its parallel parent edge's color, other edges keep theirs); writes the colors in the
 *     refined mesh's original side order to
 *     the host array colors[Ns] (the same colors dgc_refine assigned on the host) and the
 *     map kernel's time in ms (may be NULL).  Allocates its scratch, synchronises. */
dgc_status dgc_prolong_state(dgc_mesh* mesh, const double* c_coarse_dev, double* c_fine_dev, void* stream);
dgc_status dgc_restrict_state(dgc_mesh* mesh, const double* c_fine_dev, double* c_coarse_dev, void* stream);
dgc_status dgc_refine_colors_device(dgc_mesh* mesh, int8_t* colors, double* ms, void* stream);

/* Per edge (original order): the half (0: next to the coarse element's local edge's first
 * vertex, 1: the other) of the right element's local edge that a hanging edge covers, or
 * -1 for a conforming or boundary edge. */
dgc_status dgc_get_hanging(const dgc_mesh* mesh, int8_t* half);

/* Element vertex ids [E][dim+1] and unwrapped vertex coordinates [E][dim+1][dim], original
 * element order (either pointer may be NULL). */
dgc_status dgc_get_elements(const dgc_mesh* mesh, int32_t* ev, double* xyz);

/* The ordering chosen by the last coloring call: new element id of each original element,
 * new edge id of each original edge, color (1..C) of each original edge, and the color
 * offsets (C+1 entries, edges [offsets[c-1], offsets[c]) of the new order have color c).
 * Any pointer may be NULL. */
dgc_status dgc_get_ordering(const dgc_mesh* mesh, int32_t* elem_new_of_old,
                            int32_t* edge_new_of_old, int8_t* edge_color, int32_t* color_offsets);

/* Physical coordinates of each element's volume quadrature points, [E][Nq][dim], original
 * element order (unwrapped per element), and the L2 projection onto the basis of values
 * given at those points ([E][Nq][M] -> c_host [E][M][Np], original order).  Host only;
 * used to build initial states. */
dgc_status dgc_vol_points(const dgc_mesh* mesh, double* xyz);
dgc_status dgc_project(const dgc_mesh* mesh, const double* vals, double* c_host);

/* Bytes of one device state vector ([E][M][Np] FP64), and of the device workspace that
 * dgc_rk_step needs for the given precision. */
dgc_status dgc_state_size(const dgc_mesh* mesh, int64_t* bytes);
dgc_status dgc_workspace_size(const dgc_mesh* mesh, dgc_prec prec, int64_t* bytes);

/* Copy a host state (original element order, [E][M][Np] FP64) to a device state
 * (internal order), and back.  The permutation runs on the host through a pinned staging
 * buffer the mesh owns; the copy is enqueued on `stream` and the call returns after the
 * stream has completed it (it synchronises `stream`). */
dgc_status dgc_import_state(dgc_mesh* mesh, const double* c_host, double* c_dev, void* stream);
dgc_status dgc_export_state(dgc_mesh* mesh, const double* c_dev, double* c_host, void* stream);

/* Stream-ordered forms of the two calls above, for pipelines (several steps' copies in
 * flight): c_host must be pinned (page-locked or registered) host memory, xfer_dev a
 * device buffer of dgc_state_size() bytes owned by the caller (distinct per copy in
 * flight; 16-byte aligned).  Nothing is synchronised: the copy and the device permutation
 * are enqueued on `stream`, and the caller waits on the stream before touching c_host (export)
 * or reusing it (import).  DGC_ERR_ARG if c_host is not pinned. */
dgc_status dgc_import_state_async(dgc_mesh* mesh, const double* c_host, double* c_dev, double* xfer_dev,
                                  void* stream);
dgc_status dgc_export_state_async(dgc_mesh* mesh, const double* c_dev, double* c_host, double* xfer_dev,
                                  void* stream);

/* The same for the device state of a precision form: DGC_FP64 and DGC_FP32_MIXED are the
 * FP64 state above; DGC_FP32_KAHAN converts to and from its FP32 pair layout (per element,
 * mode-major with the M values of a mode together: hi and lo of the mean phi0 c0, hi of the
 * modes j >= 1, then lo of those modes; the host side stays [E][M][Np] FP64).  dgc_state_bytes gives the device bytes of either. */
dgc_status dgc_state_bytes(const dgc_mesh* mesh, dgc_prec prec, int64_t* bytes);
dgc_status dgc_import_state_prec(dgc_mesh* mesh, dgc_prec prec, const double* c_host, void* c_dev,
                                 void* stream);
dgc_status dgc_export_state_prec(dgc_mesh* mesh, dgc_prec prec, const void* c_dev, double* c_host,
                                 void* stream);

/* Right-hand side of Eq. 2: rhs_dev = dc/dt at state c_dev (FP64 rhs [E][M][Np],
 * internal order, device; c_dev in the layout of prec: FP64, or the Kahan pair state).
 * Volume integral plus the per-color surface integral of Algorithm 1 with the local
 * Lax-Friedrichs flux.  prec selects the arithmetic.  Requires a colored mesh
 * (DGC_ERR_ARG otherwise).  c_dev and rhs_dev must not alias. */
dgc_status dgc_rhs(dgc_mesh* mesh, dgc_prec prec, const void* c_dev, double* rhs_dev,
                   void* stream);

/* CFL time step, FP64, on the device:
 * dt = cfl * min_i r_i / ((2p+1) lambda_i), r_i the inradius, lambda_i the largest
 * |u| + c over element i's volume quadrature points.  Writes one double to dt_dev. */
dgc_status dgc_cfl_dt(dgc_mesh* mesh, const double* c_dev, double cfl, double* dt_dev,
                      void* stream);

/* One SSP-RK3 step (Shu-Osher form) of c_dev in place, dt from the CFL rule on the state
 * at the start of the step (written to dt_dev, device).  workspace_dev (256-byte aligned)
 * holds workspace_bytes bytes; DGC_ERR_ARG if that is less than dgc_workspace_size() for
 * prec.  The workspace also holds the step's CFL scratch, so steps of one mesh may run
 * concurrently on different streams with different workspaces and states.  No allocation and
 * no host synchronisation after the first device call on the mesh. */
dgc_status dgc_rk_step(dgc_mesh* mesh, dgc_prec prec, void* c_dev, double cfl,
                       double* dt_dev, void* workspace_dev, int64_t workspace_bytes,
                       void* stream);

/* Comparators for the race mitigation of Sec. 1 that coloring replaces.
 * dgc_rhs_atomic: one launch over all edges, contributions added with atomicAdd.
 * dgc_rhs_two_pass: every edge writes its left and right contributions to slots 2k and
 * 2k+1 of a per-edge buffer, then a per-element kernel gathers them.  buffer_dev holds
 * buffer_bytes bytes; DGC_ERR_ARG if that is less than dgc_two_pass_buffer_bytes() for
 * the mesh (FP64 words).  Same results as dgc_rhs up to rounding. */
dgc_status dgc_rhs_atomic(dgc_mesh* mesh, dgc_prec prec, const double* c_dev,
                          double* rhs_dev, void* stream);
dgc_status dgc_rhs_two_pass(dgc_mesh* mesh, dgc_prec prec, const double* c_dev,
                            double* rhs_dev, void* buffer_dev, int64_t buffer_bytes,
                            void* stream);

/* Buffer memory the per-edge two-pass scheme needs (Sec. 4.1, Table 4):
 * 2 * np * neq * sides * word_bytes. */
dgc_status dgc_two_pass_buffer_bytes(int64_t sides, int np, int neq, int word_bytes,
                                     int64_t* bytes);

/* Options (see dgc_option).  Host only. */
dgc_status dgc_set_option(dgc_mesh* mesh, dgc_option opt, int64_t value);

/* With DGC_OPT_PROFILE on: waits for the recorded events, adds the elapsed milliseconds
 * of every recorded launch to ms[class] and the launch count to launches[class]
 * (arrays of DGC_K_NCLASSES entries, zeroed by the caller), and forgets the records. */
dgc_status dgc_profile_collect(dgc_mesh* mesh, double* ms, int64_t* launches);

/* Number of kernels the last device call on this mesh enqueued. */
dgc_status dgc_last_launch_count(const dgc_mesh* mesh, int64_t* launches);

/* Batches: many independent triangle meshes of uneven size and order advanced together.
 * Each kernel class of the SSP-RK3 step (CFL passes; first / middle / last color of
 * Algorithm 1 in each stage) is ONE persistent launch over all meshes: the work is cut
 * into tiles of at most DGC_OPT_EDGES_PER_BLOCK edges (128 elements for the CFL), tiles
 * sorted by order p, each block walking tiles blockIdx, blockIdx + gridDim, ...  With
 * DGC_OPT_GRAPH (default) the 12 launches of a step are captured in a CUDA graph on the
 * first call and replayed while the buffers, precision, tile size and cfl stay the same.
 * The meshes must be colored triangle meshes in which every element has one edge of each
 * of the 3 colors (closed conforming meshes), and must outlive the batch.
 *   dgc_batch_rk_step: c_devs = host array of n device states (each [E_i][4][Np_i], FP64);
 *   dt_devs = device array of n doubles (each mesh's CFL step); workspace of
 *   dgc_batch_workspace_size() bytes, 256-byte aligned.  The first call with a new set of
 *   buffers uploads the meshes and the tile tables synchronously (make it before any
 *   capture); later calls are asynchronous.  Results equal dgc_rk_step on each mesh.
 *   dgc_batch_autotune: coordinate search over the tiles of the last, middle and first
 *   colors' launches (edges per block 16, 32, 64, 128 x threads per edge 2, or 4 in the
 *   FP32-mixed form; at most 256 threads per block), each candidate timed over 1 + reps
 *   steps -- the states advance -- keeping the fastest; the batch keeps the chosen tiles
 *   and they are written to edges_per_block[3] / threads_per_edge[3] (first, middle,
 *   last color), the best ms per step to *ms_per_step (may be NULL).
 *   DGC_OPT_EDGES_PER_BLOCK and DGC_OPT_THREADS_PER_EDGE (dgc_batch_set_option) set the
 *   tile of all three. */
dgc_status dgc_batch_create(int n, dgc_mesh* const* meshes, dgc_batch** out);
dgc_status dgc_batch_workspace_size(const dgc_batch* batch, dgc_prec prec, int64_t* bytes);
dgc_status dgc_batch_set_option(dgc_batch* batch, dgc_option opt, int64_t value);
dgc_status dgc_batch_rk_step(dgc_batch* batch, dgc_prec prec, double* const* c_devs, double cfl,
                             double* dt_devs, void* workspace_dev, int64_t workspace_bytes,
                             void* stream);
dgc_status dgc_batch_autotune(dgc_batch* batch, dgc_prec prec, double* const* c_devs, double cfl,
                              double* dt_devs, void* workspace_dev, int64_t workspace_bytes,
                              int reps, void* stream, int* edges_per_block, int* threads_per_edge,
                              double* ms_per_step);
dgc_status dgc_batch_launch_count(const dgc_batch* batch, int64_t* launches);
/* A batch's tile of one kernel class (DGC_K_FIRST, DGC_K_COLOR, DGC_K_LAST), as dgc_set_tile
 * for a mesh; threads per edge 4 applies to the FP32-mixed form (FP64 runs 2). */
dgc_status dgc_batch_set_tile(dgc_batch* batch, int kclass, int edges_per_block, int threads_per_edge);
/* With DGC_OPT_PROFILE set on the batch (dgc_batch_set_option), every step runs without its
 * graph and records a CUDA event pair on the launch stream around each launch (the reset and
 * the two CFL passes share one pair, class DGC_K_CFL; the colors are DGC_K_FIRST, DGC_K_COLOR,
 * DGC_K_LAST).  dgc_batch_profile_collect adds each class's milliseconds and event pairs since
 * the last collect into ms[] / launches[] (DGC_K_NCLASSES entries, zeroed by the caller),
 * synchronising on the events, and forgets them. */
dgc_status dgc_batch_profile_collect(dgc_batch* batch, double* ms, int64_t* launches);
void dgc_batch_destroy(dgc_batch* batch);

/* Surface-kernel tile of one kernel class of the triangle RK steps (no paper counterpart:
 * launch shape only).  kclass: DGC_K_FIRST (first color, with the volume integral),
 * DGC_K_COLOR (middle colors; also the comparators' and dgc_rhs's colors), DGC_K_LAST
 * (last color with the stage update).  edges_per_block 16..128 (a multiple of 16),
 * threads_per_edge 2 or 4 (4: triangle meshes, FP32 forms of dgc_rk_step /
 * dgc_rk_step_static; two lanes per edge side split the edge's quadrature points, the
 * volume integral's points and the epilogue's modes), at most 256 threads per block;
 * else DGC_ERR_ARG (DGC_ERR_UNSUPPORTED for 4 on other element types).  The options
 * DGC_OPT_EDGES_PER_BLOCK / DGC_OPT_THREADS_PER_EDGE set all three classes. */
dgc_status dgc_set_tile(dgc_mesh* mesh, int kclass, int edges_per_block, int threads_per_edge);
dgc_status dgc_get_tile(const dgc_mesh* mesh, int kclass, int* edges_per_block, int* threads_per_edge);

/* Tile autotuner for one mesh's RK step: coordinate search over the last, middle and
 * first colors' tiles (edges per block 32 / 64 / 128 x threads per edge 2 / 4 where
 * allowed), each candidate timed over `reps` steps (after one untimed step) with CUDA
 * events on `stream`, keeping the fastest; the mesh keeps the chosen tiles.  The steps
 * advance c_dev (pass a scratch copy of the state).  Writes the tiles of FIRST, COLOR,
 * LAST into edges_per_block[3] / threads_per_edge[3] and the best time per step (ms, may
 * be NULL).  Arguments as dgc_rk_step. */
dgc_status dgc_autotune(dgc_mesh* mesh, dgc_prec prec, void* c_dev, double cfl, double* dt_dev,
                        void* workspace_dev, int64_t workspace_bytes, int reps, void* stream,
                        int* edges_per_block, int* threads_per_edge, double* ms_per_step);

/* Thread-local message of the last error (empty string if none). */
const char* dgc_last_error(void);

/* dgc_rk_step for callers that cannot allocate device memory: the same SSP-RK3 step
 * (same kernels, same results), but the workspace and the CFL scratch are taken from a
 * 16 MiB array the library holds in device memory, so the caller passes no workspace and
 * the call allocates nothing (no cudaMalloc, cudaFree or allocating library call).  It
 * serves callers whose device memory is owned by someone else -- a host framework that
 * reserves the whole device for its own pool, or a fixed-footprint solver loop that may
 * not change its allocations once running -- and so cannot produce the workspace
 * dgc_rk_step needs.  The paper has no counterpart; this is an interface addition.
 *   Limits: dgc_workspace_size(mesh, prec) must not exceed 16 MiB (16,777,216 bytes):
 *   e.g. up to about 24,800 triangles at p = 3 and 73,500 at p = 1 in the FP32-mixed
 *   form, 26,000 and 85,500 in FP64; larger meshes get DGC_ERR_ARG.  The mesh must already be
 *   on the current device from an earlier device call (uploading allocates), else
 *   DGC_ERR_ARG.
 *   When the 16 MiB is reserved: at the first mesh upload on each device (the first
 *   device call on a mesh: dgc_import_state, dgc_rhs, dgc_cfl_dt, dgc_rk_step, ...),
 *   which loads the library's module holding the array; from then on every such GPU
 *   holds it until the process exits, and this call only reads its cached address.
 *   (Under the CUDA driver's lazy module loading, each kernel's code is still loaded on
 *   its first launch; a caller that fixes its footprint makes one step first.)
 *   The array is shared by every call on a device and keeps the last call's contents
 *   (each call writes what it reads first; dt_dev and the CFL minimum are reset per call).
 *   Calls whose work overlaps on the GPU (two streams, or two meshes at once) race on
 *   the array: serialise them.  A context reset (cudaDeviceReset) frees the array with
 *   every other device buffer of the library: destroy the meshes before one; the next mesh
 *   upload on the new context looks the array up again. */
dgc_status dgc_rk_step_static(dgc_mesh* mesh, dgc_prec prec, void* c_dev, double cfl,
                              double* dt_dev, void* stream);

/* Free the mesh and its device copies (the device must still be current). */
void dgc_destroy(dgc_mesh* mesh);

#ifdef __cplusplus
}
#endif

#endif /* DGC_H */
