// Device-side declarations shared by the C ABI (capi.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dgc_internal.h"

namespace dgc {

// A boundary face's left-element first vertex and edge vector (the shock's points).
struct BndGeo {
  double x0, y0, dx, dy;
};

// Device copies of one mesh, in the internal (renumbered) order.
struct DeviceMesh {
  int device = -1;
  double* jinv = nullptr;   // [E][dim*dim] rows = gradients of the reference coordinates
  double* inr = nullptr;    // [E] inradius
  // [Ns] (left, right or -1, lq | rq << 4 | orient << 8, 0).  On triangles rq is
  // the right element's edge table: its local edge 0..2, or 3 + 2 f + h for
  // half h of local edge f (coarse side of a hanging edge), 15 on a boundary
  int4* topo = nullptr;
  double2* fgeo = nullptr;  // [Ns][2] 2D: (nx, ny), (|f|/detJ_l, |f|/detJ_r); 3D: [Ns][3]
  int32_t* slots = nullptr; // [E][slot_w] two-pass gather slots 2k + side, -1 unused
  int slot_w = 3;           // sides per element at most (nfpe; 2 nfpe when refined)
  int edge_tables = 3;      // triangle edge tables the surface kernels stage (3, or 9 when refined)
  float* ftab = nullptr;    // 3D face tables (float copy)
  double* ftabd = nullptr;  // 3D face tables
  float2* ftabdf = nullptr; // 3D face tables as FP32 pairs (hi, lo): the FP64 kernels
  float2* vtabdf = nullptr; // 3D volume tables as FP32 pairs [4][NQV][NP]: the FP64 kernels
  float* cfl_est = nullptr; // [E] FP32 step estimates of the CFL pre-pass, then 1 minimum
  int32_t* perm = nullptr;  // [E] internal element id of each original element (import / export)
  double* xfer = nullptr;   // [E][M*Np] state in original order (import / export; allocated on first use)
  // refined meshes: state transfer to and from the mesh before refinement
  // (internal orders): per fine element its coarse element and child 0..3 (4:
  // copy), per coarse element its children's fine ids (kids[1] = -1: one copy),
  // and the child projections P [4][Np][Np]
  // hybrid triangle/quadrilateral meshes: per element its kind (0 triangle, 1
  // quadrilateral), and the tables of kernels_hybrid.cu
  int8_t* hyb_kind = nullptr;  // 2: a general (bilinear) quadrilateral
  double* hyb_tab = nullptr;
  // general quadrilaterals: per element its slot (-1: none), and per slot
  // detJ J^-1 at the volume points [NQV][4] and the inverse mass matrix [Np][Np]
  int32_t* bil_slot = nullptr;
  int32_t* bil_elem = nullptr;
  double* bil_G = nullptr;
  double* bil_Minv = nullptr;
  int64_t nbil = 0;
  // boundary conditions (dgc_set_boundary; null: every boundary transmissive):
  // the boundary block (kBc*), per boundary face (the index in topo.w >> 8) the
  // left element's first vertex of the face and the edge vector (x0, y0, dx,
  // dy), the time the boundary states are taken at (advanced by each RK step)
  double* bc = nullptr;
  BndGeo* bgeo = nullptr;
  double* time = nullptr;
  // the limiter: per element its face neighbours (-1 on a boundary), internal ids
  int4* enb = nullptr;
  int32_t* xf_src = nullptr;
  int8_t* xf_kind = nullptr;
  int32_t* xf_kids = nullptr;
  double* xf_P = nullptr;
};

// The boundary block: up to kBcMaxStates prescribed states [4] from kBcStates,
// then the shock's a, b, c and its states behind and ahead (as doubles).
constexpr int kBcMaxStates = 8, kBcStates = 0, kBcShock = 4 * kBcMaxStates, kBcDoubles = kBcShock + 8;

// Surface-kernel modes (Algorithm 1 and the comparators of Sec. 1).
enum SurfMode {
  SURF_RMW = 0,     // add into rhs (colors after the first)
  SURF_FIRST = 1,   // volume integral + surface, plain store (first color, closed meshes)
  SURF_ATOMIC = 2,  // atomicAdd into rhs (comparator)
  SURF_BUFFER = 3,  // write per-edge buffer slots 2k, 2k+1 (comparator)
  SURF_LAST = 4     // last color: finish rhs in registers and apply the RK stage update
};

// Type configurations: storage of the state read, compute type, rhs type.
enum TypeCfg {
  TY_D = 0,     // FP64 state, FP64 arithmetic, FP64 rhs
  TY_MD = 1,    // FP64 state, FP32 arithmetic, FP64 rhs (dgc_rhs in mixed precision)
  TY_MF = 2,    // FP32 record, FP32 arithmetic, FP32 rhs (RK stages of the FP32 forms)
  TY_KD = 3     // FP32 record (Kahan state), FP32 arithmetic, FP64 rhs (dgc_rhs, Kahan form)
};

// FP32 record of the state kept by the mixed-precision step: rec floats per
// element; split = the mean state phi0 c0 stored as an FP32 pair (hi[M], lo[M])
// followed by the modes j >= 1 as [M][np-1], padded to rec floats; otherwise a
// plain FP32 copy of the M*np values.
struct ShadowLayout {
  int M = 4, np = 1, nv = 4, rec = 4;
  bool split = false;
  bool mode_major = false;  // FP32 buffers as [NP][M] (triangles), else [M][NP]
  double phi0 = 0.0;
};

struct Ctx {
  int dim = 2, p = 1, np = 0, M = 4, nfpe = 3;
  bool quad = false;  // quadrilateral mesh (kernels_quad.cu)
  ShadowLayout shadow;
  int64_t ne = 0, ns = 0;
  int epb = 128;
  // triangle kernels: edges per block and threads per edge (2: one lane per
  // edge side; 4: two lanes per side, FP32 right-hand sides of an RK step) of
  // the first, middle and last colors
  int tile_epb[3] = {128, 128, 128};
  int tile_tpe[3] = {2, 2, 2};
  // triangle surface kernels: grid-stride over the color with one wave of
  // blocks (sms = the GPU's multiprocessors) instead of one block per tile
  bool persistent = false;
  int sms = 0;
  bool hybrid = false;  // hybrid triangle/quadrilateral mesh: kernels_hybrid.cu (FP64)
  const DeviceMesh* d = nullptr;
  cudaStream_t st = nullptr;
  bool pdl = false;  // launch the surface and CFL kernels with programmatic dependent launch
  // the time boundary states are taken at: the mesh's time + tfrac * (*dtp)
  // (the RK stages: 0, 1, 1/2 of the step's dt; dtp null: the mesh's time)
  double tfrac = 0.0;
  const double* dtp = nullptr;
};

// A kernel launch on x.st with smem bytes of dynamic shared memory; with x.pdl,
// as a programmatic dependent launch (the kernels pair pdl_wait / pdl_trigger,
// dev_util.cuh).
template <typename... KArgs, typename... Args>
static void launch_k(const Ctx& x, void (*k)(KArgs...), unsigned grid, unsigned threads, size_t smem, Args... args) {
  if (!x.pdl) {
    k<<<grid, threads, smem, x.st>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = x.st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);
}

struct StageArgs {
  // FP64 form: uout = a0 u0 + b0 (us + dt L(us))
  const double* u0 = nullptr;  // FP64 state at the start of the step
  double* uout = nullptr;      // FP64 stage output (may alias the stage input)
  const double* dt = nullptr;  // device time step
  double a0 = 0.0, b0 = 1.0;
  // FP32 forms, increment form of the step (incr_form.cuh)
  int stage = 0;                // 0, 1, 2
  const float* rec0 = nullptr;  // FP32 record of u0 (the Kahan state itself in the Kahan form)
  int rec0_stride = 0;          // floats per element of rec0
  float* rec_out = nullptr;     // FP32 record of the next stage's state (stages 0, 1)
  float* delta = nullptr;       // [E][M*Np] stage increment
  float* kstate = nullptr;      // Kahan form: the FP32 pair state (stride rec0_stride); else null
};

// One mesh of a batch, as the batched kernels see it (device array).
struct BatchMeshDev {
  int p = 0, pad = 0;
  int64_t ne = 0;
  const int4* topo = nullptr;
  const double2* fgeo = nullptr;
  const double* jinv = nullptr;
  const double* inr = nullptr;
  float* est = nullptr;   // CFL estimates [ne], minimum at [ne]
  double* c = nullptr;    // state (caller's)
  double* u1 = nullptr;   // FP64 stage state (workspace, FP64 form)
  float* rec0 = nullptr;  // FP32 record of u0 (workspace, mixed precision)
  float* recs = nullptr;  // FP32 record of the stage state (workspace, mixed precision)
  float* delta = nullptr; // FP32 stage increment (workspace, mixed precision)
  void* rhs = nullptr;    // rhs (workspace)
  double* dt = nullptr;   // this mesh's time step (caller's)
};

// A range of one mesh's edges (of one color) or elements, at most one block's work.
struct BatchTile {
  int32_t mesh = 0, p = 0;
  int64_t begin = 0, end = 0;
};

// kernels_tri.cu
void tri_upload_tables(int p, const RefTables& T);
int batch_init(cudaStream_t st, const BatchMeshDev* d, int n);
int batch_cfl(cudaStream_t st, const BatchMeshDev* d, const BatchTile* tiles, int nt, double cfl, bool mixed);
int batch_surf(cudaStream_t st, const BatchMeshDev* d, const BatchTile* tiles, int nt, int stage, double a0,
               double b0, SurfMode mode, bool mixed, int threads, int tpe);
int tri_record_floats(int p);
// sstride: floats per element of an FP32 state (record or Kahan state); ignored for FP64 states
// volume kernels cover elements [e0, ne)
int tri_volume(const Ctx& c, TypeCfg ty, const void* state, int sstride, void* rhs, int64_t e0 = 0);
// hybrid triangle/quadrilateral meshes, FP64 (kernels_hybrid.cu): the volume
// integral of every element (plain store), one color's edges (read-modify-write,
// or atomics), the CFL step into *dt; the table size in doubles
// fp32: the FP32-mixed kernels (FP32 flux and projection, FP64 state and rhs)
int hyb_volume(const Ctx& x, const double* state, double* rhs, bool fp32 = false);
int hyb_surface(const Ctx& x, bool atomic, int64_t begin, int64_t end, const double* state, double* rhs,
                bool fp32 = false);
int hyb_cfl(const Ctx& x, const double* state, double cfl, double* dt);
// general quadrilaterals: rhs <- M^-1 rhs on every bilinear element
int hyb_mass(const Ctx& x, double* rhs);
int hyb_table_doubles(int p);
// dgc_rhs of a triangle mesh in one cooperative launch (FP64 or FP32-mixed with
// FP64 state and rhs): off = the color offsets, fused = the first color also
// stores the volume integral of the elements [0, e_vol0)
int tri_rhs_coop(const Ctx& x, TypeCfg ty, const int* off, int ncolors, bool fused, int64_t e_vol0,
                 const void* state, void* rhs);
int tri_surface(const Ctx& c, TypeCfg ty, SurfMode mode, int64_t begin, int64_t end, const void* state,
                int sstride, void* rhs, void* buf, const StageArgs* sa);
int tri_cfl(const Ctx& c, const double* state, double cfl, double* dt, float* shadow);
// the limiter on an FP64 triangle state, in place (kernels_tri.cu k_limit_tri)
int tri_limit(const Ctx& x, double* c);
// the mesh's device time += *dt (meshes with boundary conditions)
int time_advance(const Ctx& x, const double* dt);
// stage 0 of the mixed step on perfectly colored meshes: the first color also
// writes the record of u0 and the CFL estimates (pass 1); pass 2 alone
int tri_first_est(const Ctx& c, int64_t begin, int64_t end, const double* state, float* rec0, float* rhs);
int tri_cfl_pass2(const Ctx& c, const double* state, double cfl, double* dt);
int tri_kahan_floats(int p);
int tri_cfl_kahan(const Ctx& c, const float* kstate, double cfl, double* dt);

// kernels_tet.cu
void tet_upload_tables(int p, const RefTables& T, DeviceMesh& d);
int tet_record_floats(int p);
int tet_volume(const Ctx& c, TypeCfg ty, const void* state, int sstride, void* rhs, int64_t e0 = 0);
int tet_surface(const Ctx& c, TypeCfg ty, SurfMode mode, int64_t begin, int64_t end, const void* state,
                int sstride, void* rhs, void* buf, const StageArgs* sa);
int tet_cfl(const Ctx& c, const double* state, double cfl, double* dt, float* shadow);

// kernels_quad.cu
void quad_upload_tables(int p, const RefTables& T);
int quad_record_floats(int p);
int quad_volume(const Ctx& c, TypeCfg ty, const void* state, int sstride, void* rhs, int64_t e0 = 0);
int quad_surface(const Ctx& c, TypeCfg ty, SurfMode mode, int64_t begin, int64_t end, const void* state,
                 int sstride, void* rhs, void* buf, const StageArgs* sa);
int quad_cfl(const Ctx& c, const double* state, double cfl, double* dt, float* shadow);

// kernels_common.cu
int stage_update(const Ctx& c, bool rhs_f32, const double* us, const void* rhs, const StageArgs& sa);
int incr_stage_update(const Ctx& c, const float* rhs, const StageArgs& sa);
int gather_two_pass(const Ctx& c, bool f32, void* rhs, const void* buf);
// element blocks of nv doubles between original and internal order:
// to_internal: dst[perm[e]] = src[e]; else dst[e] = src[perm[e]]
// refinement on the device (kernels_common.cu): the Sec. 3.2 color map of the
// refined sides, and the state between a mesh and its refinement (prolong: n =
// fine elements, src / kind per fine element; restrict: n = coarse elements,
// kids[4] per coarse element; P [4][NP][NP])
int refine_colors(cudaStream_t st, const int8_t* base_color, const int32_t* base_face_of, const int32_t* src,
                  const int8_t* rule, int64_t ns, int8_t* out);
int transfer_state(cudaStream_t st, bool prolong, const double* in, double* out, const int32_t* src,
                   const int8_t* kind, const int32_t* kids, const double* P, int64_t n, int M, int NP);
int permute_blocks(cudaStream_t st, double* dst, const double* src, const int32_t* perm, int nv, int64_t ne,
                   bool to_internal);

}  // namespace dgc
