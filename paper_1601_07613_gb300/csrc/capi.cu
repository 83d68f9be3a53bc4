// C ABI of the library (include/dgc.h): argument checks, device upload of the
// renumbered mesh, and the launch sequences of Algorithm 1 and SSP-RK3.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <set>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "device.cuh"

using namespace dgc;

namespace {

thread_local std::string g_err;

#define DGC_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError(); /* a failed call leaves its code pending; do not report it twice */ \
      throw Error{DGC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};        \
    }                                                                                       \
  } while (0)

template <typename F>
dgc_status guarded(F&& f) {
  try {
    f();
    g_err.clear();
    return DGC_OK;
  } catch (const Error& e) {
    g_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return DGC_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return DGC_ERR_ARG;
  }
}

void require(bool ok, const char* msg, dgc_status code = DGC_ERR_ARG) {
  if (!ok) throw Error{code, msg};
}

int64_t nv_of(const Mesh& m) { return (int64_t)m.M * m.np; }
// floats per element of the FP32 record the mixed-precision step keeps
int64_t record_floats(const Mesh& m) {
  return m.quad ? quad_record_floats(m.p) : m.dim == 2 ? tri_record_floats(m.p) : tet_record_floats(m.p);
}
// floats per element of the FP32 pair state of the Kahan form (triangles)
int64_t kahan_floats(const Mesh& m) { return tri_kahan_floats(m.p); }
int64_t state_bytes(const Mesh& m) { return m.ne * nv_of(m) * (int64_t)sizeof(double); }
int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

// host staging buffer (pinned) used by import / export
struct Staging {
  double* ptr = nullptr;
  int64_t bytes = 0;
};
std::mutex g_stage_mu;
std::vector<std::pair<const Mesh*, Staging>> g_staging;

double* staging_for(const Mesh& m) {
  std::lock_guard<std::mutex> lk(g_stage_mu);
  for (size_t i = 0; i < g_staging.size(); ++i)
    if (g_staging[i].first == &m) {
      if (g_staging[i].second.bytes >= state_bytes(m)) return g_staging[i].second.ptr;
      cudaFreeHost(g_staging[i].second.ptr);  // the mesh grew (refinement): a larger buffer
      g_staging.erase(g_staging.begin() + i);
      break;
    }
  Staging s;
  s.bytes = state_bytes(m);
  DGC_CUDA(cudaMallocHost(&s.ptr, s.bytes));
  g_staging.emplace_back(&m, s);
  return s.ptr;
}

void staging_free(const Mesh& m) {
  std::lock_guard<std::mutex> lk(g_stage_mu);
  for (size_t i = 0; i < g_staging.size(); ++i)
    if (g_staging[i].first == &m) {
      cudaFreeHost(g_staging[i].second.ptr);
      g_staging.erase(g_staging.begin() + i);
      return;
    }
}

template <typename F>
void parallel_for(int64_t n, F&& f) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (n < 4096 || nt == 1) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b < e) th.emplace_back([&f, b, e] { f(b, e); });
  }
  for (auto& t : th) t.join();
}

std::mutex g_tab_mu;
std::set<std::pair<int, int>> g_tab_done;  // (device, dim*16 + p)

// Device address of the allocation-free step's static array on device dev
// (defined with the step below).  load = true looks it up on first use, which
// loads the module that holds the array and so reserves its device memory;
// load = false only returns the address cached by an earlier lookup.
void* static_scratch(int dev, bool load);

template <typename T>
T* dalloc(int64_t n) {
  T* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(T) * std::max<int64_t>(n, 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{e == cudaErrorMemoryAllocation ? DGC_ERR_OOM : DGC_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  }
  return p;
}

// Hybrid meshes: each element's kind (internal order) and the tables of
// kernels_hybrid.cu: per kind (triangle, quadrilateral) the basis and the
// weighted reference gradients at the (p+1)^2 volume points and the basis at the
// 2p+1 Gauss points of each local edge (from its first vertex to its second),
// zero past the kind's modes, then the edge weights (summing to 1).
void upload_hybrid(const Mesh& m, DeviceMesh& d) {
  const int p = m.p, NPX = m.np, NQE = 2 * p + 1;
  const int NQV = m.tab.nqv;
  const int VOL = NQV * NPX, EDGE = 4 * NQE * NPX;
  std::vector<double> t((size_t)hyb_table_doubles(p), 0.0);
  if ((int64_t)t.size() != 2 * (3 * VOL + EDGE) + NQE || m.tab_tri.nqv != NQV)
    throw Error{DGC_ERR_UNSUPPORTED, "hybrid meshes: p = 1..3"};
  std::vector<double> xg(NQE), wg(NQE);
  gauss_jacobi(NQE, 0.0, xg.data(), wg.data());
  const double refv[2][4][2] = {{{0, 0}, {1, 0}, {0, 1}, {0, 0}}, {{0, 0}, {1, 0}, {1, 1}, {0, 1}}};
  for (int k = 0; k < 2; ++k) {
    const RefTables& T = k ? m.tab : m.tab_tri;
    const int np = T.np, nf = k ? 4 : 3;
    double* vol = &t[(size_t)k * 3 * VOL];
    for (int q = 0; q < NQV; ++q)
      for (int j = 0; j < np; ++j) {
        vol[q * NPX + j] = T.phiV[(size_t)q * np + j];
        vol[VOL + q * NPX + j] = T.vw[q] * T.dphiV[(size_t)q * np + j];
        vol[2 * VOL + q * NPX + j] = T.vw[q] * T.dphiV[((size_t)NQV + q) * np + j];
      }
    double* edge = &t[(size_t)6 * VOL + (size_t)k * EDGE];
    std::vector<double> phi(np);
    for (int f = 0; f < nf; ++f)
      for (int q = 0; q < NQE; ++q) {
        const double tq = 0.5 * (1.0 + xg[q]);
        const double* A = refv[k][f];
        const double* B = refv[k][(f + 1) % nf];
        const double x[2] = {A[0] + tq * (B[0] - A[0]), A[1] + tq * (B[1] - A[1])};
        basis_eval(2, p, x, phi.data(), nullptr, k == 1);
        for (int j = 0; j < np; ++j) edge[((size_t)f * NQE + q) * NPX + j] = phi[j];
      }
  }
  for (int q = 0; q < NQE; ++q) t[(size_t)6 * VOL + 2 * EDGE + q] = 0.5 * wg[q];
  std::vector<int8_t> kind(m.ne);
  std::vector<int32_t> slot(m.ne, -1), belem;
  std::vector<double> G, Mi;
  int64_t nb = 0;
  for (int64_t e = 0; e < m.ne; ++e) {
    const int32_t n = m.elem_new_of_old[e];
    const bool bil = !m.bil.empty() && m.bil[e];
    kind[n] = bil ? 2 : (int8_t)(m.ev[(size_t)e * 4 + 3] >= 0);
    if (!bil) continue;
    slot[n] = (int32_t)nb++;
    belem.push_back(n);
    const double* X = &m.X[(size_t)e * 8];
    for (int q = 0; q < NQV; ++q) {  // detJ J^-1 (rows: gradients of r and s) at the point
      double J[4];
      bilinear_map(X, m.tab.vr[q], m.tab.vs[q], nullptr, J);
      G.insert(G.end(), {J[3], -J[1], -J[2], J[0]});
    }
    const std::vector<double> inv = bilinear_mass_inverse(m, e);
    Mi.insert(Mi.end(), inv.begin(), inv.end());
  }
  d.hyb_kind = dalloc<int8_t>(m.ne);
  d.hyb_tab = dalloc<double>((int64_t)t.size());
  DGC_CUDA(cudaMemcpy(d.hyb_kind, kind.data(), kind.size(), cudaMemcpyHostToDevice));
  DGC_CUDA(cudaMemcpy(d.hyb_tab, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice));
  d.nbil = nb;
  if (nb > 0) {
    d.bil_slot = dalloc<int32_t>(m.ne);
    d.bil_elem = dalloc<int32_t>(nb);
    DGC_CUDA(cudaMemcpy(d.bil_elem, belem.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
    d.bil_G = dalloc<double>((int64_t)G.size());
    d.bil_Minv = dalloc<double>((int64_t)Mi.size());
    DGC_CUDA(cudaMemcpy(d.bil_slot, slot.data(), sizeof(int32_t) * slot.size(), cudaMemcpyHostToDevice));
    DGC_CUDA(cudaMemcpy(d.bil_G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice));
    DGC_CUDA(cudaMemcpy(d.bil_Minv, Mi.data(), sizeof(double) * Mi.size(), cudaMemcpyHostToDevice));
  }
}

// Refined triangle meshes: the tables of the state transfer to and from the
// mesh before refinement (internal orders of both), and the child projections
// P_c[j][k] = sum_q w_q phi_j(rho_q) phi_k(A_c rho_q) of the reference triangle
// (A_c: child c's reference triangle inside its parent's, children ordered as
// refine() makes them: [v0, m01, m20], [m01, v1, m12], [m20, m12, v2],
// [m01, m12, m20]); the volume rule integrates the degree-2p products exactly.
void upload_transfer(const Mesh& m, DeviceMesh& d) {
  const Mesh::Base& b = m.base;
  const int np = m.np;
  std::vector<int32_t> src(m.ne, -1), kids((size_t)b.ne * 4, -1);
  std::vector<int8_t> kind(m.ne, 4);
  for (int64_t e = 0, n = 0; e < b.ne; ++e) {
    const int32_t ce = b.elem_new_of_old[e];
    const int k = b.flag[e] ? 4 : 1;
    for (int c = 0; c < k; ++c, ++n) {
      const int32_t fe = m.elem_new_of_old[n];
      src[fe] = ce;
      kind[fe] = (int8_t)(k == 4 ? c : 4);
      kids[(size_t)ce * 4 + c] = fe;
    }
  }
  // A_c (rho, sigma) = o + a rho + b sigma in the parent's reference coordinates
  const double A[4][6] = {{0.0, 0.0, 0.5, 0.0, 0.0, 0.5},
                          {0.5, 0.0, 0.5, 0.0, 0.0, 0.5},
                          {0.0, 0.5, 0.5, 0.0, 0.0, 0.5},
                          {0.5, 0.0, 0.0, 0.5, -0.5, 0.5}};
  std::vector<double> P((size_t)4 * np * np, 0.0), phi(np), phic(np);
  for (int c = 0; c < 4; ++c)
    for (int q = 0; q < m.tab.nqv; ++q) {
      const double x[2] = {m.tab.vr[q], m.tab.vs[q]};
      const double y[2] = {A[c][0] + A[c][2] * x[0] + A[c][4] * x[1], A[c][1] + A[c][3] * x[0] + A[c][5] * x[1]};
      basis_eval(2, m.p, x, phic.data(), nullptr);
      basis_eval(2, m.p, y, phi.data(), nullptr);
      for (int j = 0; j < np; ++j)
        for (int k = 0; k < np; ++k) P[((size_t)c * np + j) * np + k] += m.tab.vw[q] * phic[j] * phi[k];
    }
  d.xf_src = dalloc<int32_t>(m.ne);
  d.xf_kind = dalloc<int8_t>(m.ne);
  d.xf_kids = dalloc<int32_t>((int64_t)kids.size());
  d.xf_P = dalloc<double>((int64_t)P.size());
  DGC_CUDA(cudaMemcpy(d.xf_src, src.data(), sizeof(int32_t) * src.size(), cudaMemcpyHostToDevice));
  DGC_CUDA(cudaMemcpy(d.xf_kind, kind.data(), kind.size(), cudaMemcpyHostToDevice));
  DGC_CUDA(cudaMemcpy(d.xf_kids, kids.data(), sizeof(int32_t) * kids.size(), cudaMemcpyHostToDevice));
  DGC_CUDA(cudaMemcpy(d.xf_P, P.data(), sizeof(double) * P.size(), cudaMemcpyHostToDevice));
}

// Upload the renumbered mesh: per element inverse Jacobian and inradius, per
// edge (new order) its elements, local faces, normal and |f|/detJ factors,
// and the two-pass gather slots.
void upload(Mesh& m) {
  int dev = -1;
  DGC_CUDA(cudaGetDevice(&dev));
  if (m.dev && m.dev->device != dev) throw Error{DGC_ERR_ARG, "mesh was uploaded on another device"};
  if (m.dev && !m.dirty) return;
  device_free(m);
  const int dim = m.dim, nfpe = m.nfpe;
  const std::vector<int32_t>& en = m.elem_new_of_old;
  std::vector<double> jinv((size_t)m.ne * dim * dim), inr(m.ne);
  for (int64_t e = 0; e < m.ne; ++e) {
    int64_t n = en[e];
    std::copy_n(&m.Jinv[(size_t)e * dim * dim], dim * dim, &jinv[(size_t)n * dim * dim]);
    inr[n] = m.inradius[e];
  }
  const int gstride = dim == 2 ? 2 : 3;  // double2 per edge
  std::vector<int4> topo(m.ns);
  std::vector<double2> fgeo((size_t)m.ns * gstride);
  const int slot_w = m.refined ? 2 * nfpe : nfpe;
  std::vector<int32_t> slots((size_t)m.ne * slot_w, -1);
  std::vector<BndGeo> bgeo;  // boundary conditions: per boundary face its first vertex and edge vector
  for (int64_t k = 0; k < m.ns; ++k) {
    int64_t old = m.side_old_of_new[k];
    int32_t l = m.sl[old], r = m.sr[old];
    const int h = m.shalf.empty() ? -1 : m.shalf[old];
    int ql = m.sql[old], qr = r < 0 ? 15 : (h >= 0 ? 3 + 2 * m.sqr[old] + h : m.sqr[old]);
    int orient = 0;
    if (dim == 3 && r >= 0) {
      // vertex permutation between the two sides' face parameterisations:
      // vertex i of the right element's face is vertex perm[i] of the left's
      int32_t gl[3], gr[3], n = 0;
      for (int v = 0, a = 0, b = 0; v < 4; ++v) {
        if (v != ql) gl[a++] = m.ev[(size_t)l * 4 + v];
        if (v != qr) gr[b++] = m.ev[(size_t)r * 4 + v];
      }
      int perm[3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          if (gr[i] == gl[j]) perm[i] = j, ++n;
      orient = -1;
      for (int o = 0; o < 6 && n == 3; ++o)
        if (kFacePerms[o][0] == perm[0] && kFacePerms[o][1] == perm[1] && kFacePerms[o][2] == perm[2]) orient = o;
      if (orient < 0) throw Error{DGC_ERR_MESH, "face vertices of the two sides do not match"};
    }
    int bw = 0;  // boundary conditions: kind | state << 4 | boundary face << 8
    if (m.has_bc && r < 0) {
      bw = m.bc_kind[old] | (m.bc_sidx[old] << 4) | ((int)bgeo.size() << 8);
      const double* X = &m.X[(size_t)l * 6];
      const double* A = X + 2 * ql;
      const double* B = X + 2 * ((ql + 1) % 3);
      bgeo.push_back(BndGeo{A[0], A[1], B[0] - A[0], B[1] - A[1]});
    }
    topo[k] = make_int4(en[l], r >= 0 ? en[r] : -1, ql | (qr << 4) | (orient << 8), bw);
    double meas = m.smeas[old];
    // |f| / detJ per side (a bilinear element's detJ varies: its mass matrix is
    // applied after the colors instead, so its factor is |f|)
    auto fdet = [&](int32_t e) { return m.bil.empty() || !m.bil[e] ? m.detJ[e] : 1.0; };
    double sl = meas / fdet(l), sr = r >= 0 ? meas / fdet(r) : 0.0;
    const double* n = &m.snormal[(size_t)old * dim];
    if (dim == 2) {
      fgeo[2 * k] = make_double2(n[0], n[1]);
      fgeo[2 * k + 1] = make_double2(sl, sr);
    } else {
      fgeo[3 * k] = make_double2(n[0], n[1]);
      fgeo[3 * k + 1] = make_double2(n[2], 0.0);
      fgeo[3 * k + 2] = make_double2(sl, sr);
    }
    slots[(size_t)en[l] * slot_w + ql] = (int32_t)(2 * k);
    if (r >= 0) {
      const int q = m.sqr[old];
      int32_t* sr_ = &slots[(size_t)en[r] * slot_w];
      sr_[sr_[q] < 0 ? q : nfpe + q] = (int32_t)(2 * k + 1);
    }
  }
  auto d = std::make_unique<DeviceMesh>();
  d->device = dev;
  d->slot_w = slot_w;
  d->edge_tables = m.refined ? 9 : 3;
  try {
    d->jinv = dalloc<double>((int64_t)jinv.size());
    d->inr = dalloc<double>(m.ne);
    d->topo = dalloc<int4>(m.ns);
    d->fgeo = dalloc<double2>((int64_t)fgeo.size());
    d->slots = dalloc<int32_t>((int64_t)slots.size());
    d->cfl_est = dalloc<float>(m.ne + 64);
    d->perm = dalloc<int32_t>(m.ne);
    DGC_CUDA(cudaMemcpy(d->perm, en.data(), sizeof(int32_t) * m.ne, cudaMemcpyHostToDevice));
    DGC_CUDA(cudaMemcpy(d->jinv, jinv.data(), sizeof(double) * jinv.size(), cudaMemcpyHostToDevice));
    DGC_CUDA(cudaMemcpy(d->inr, inr.data(), sizeof(double) * inr.size(), cudaMemcpyHostToDevice));
    DGC_CUDA(cudaMemcpy(d->topo, topo.data(), sizeof(int4) * topo.size(), cudaMemcpyHostToDevice));
    DGC_CUDA(cudaMemcpy(d->fgeo, fgeo.data(), sizeof(double2) * fgeo.size(), cudaMemcpyHostToDevice));
    DGC_CUDA(cudaMemcpy(d->slots, slots.data(), sizeof(int32_t) * slots.size(), cudaMemcpyHostToDevice));
    if (dim == 3) tet_upload_tables(m.p, m.tab, *d);
    if (m.quad) quad_upload_tables(m.p, m.tab);
    if (m.refined) upload_transfer(m, *d);
    if (m.hybrid) upload_hybrid(m, *d);
    if (m.has_bc) {
      std::vector<double> blk(kBcDoubles, 0.0);
      std::copy(m.bc_states.begin(), m.bc_states.end(), blk.begin() + kBcStates);
      for (int a = 0; a < 3; ++a) blk[kBcShock + a] = m.shock[a];
      blk[kBcShock + 3] = m.shock_st[0];
      blk[kBcShock + 4] = m.shock_st[1];
      d->bc = dalloc<double>(kBcDoubles);
      DGC_CUDA(cudaMemcpy(d->bc, blk.data(), sizeof(double) * blk.size(), cudaMemcpyHostToDevice));
      d->bgeo = dalloc<BndGeo>(std::max<int64_t>(1, (int64_t)bgeo.size()));
      if (!bgeo.empty())
        DGC_CUDA(cudaMemcpy(d->bgeo, bgeo.data(), sizeof(BndGeo) * bgeo.size(), cudaMemcpyHostToDevice));
    }
    if (dim == 2 && !m.quad) {
      // the mesh's time (boundary states) and the limiter's face neighbours
      d->time = dalloc<double>(1);
      DGC_CUDA(cudaMemcpy(d->time, &m.time, sizeof(double), cudaMemcpyHostToDevice));
      if (!m.refined && m.want_enb) {
        std::vector<int4> enb(m.ne);
        for (int64_t e = 0; e < m.ne; ++e) {
          int nb[3];
          for (int f = 0; f < 3; ++f) {
            const int32_t sd = m.face_of[(size_t)e * 3 + f];
            const int32_t o = sd < 0 ? -1 : (m.sl[sd] == e ? m.sr[sd] : m.sl[sd]);
            nb[f] = o < 0 ? -1 : en[o];
          }
          enb[en[e]] = make_int4(nb[0], nb[1], nb[2], 0);
        }
        d->enb = dalloc<int4>(m.ne);
        DGC_CUDA(cudaMemcpy(d->enb, enb.data(), sizeof(int4) * enb.size(), cudaMemcpyHostToDevice));
      }
    }
  } catch (...) {
    m.dev = d.release();
    device_free(m);
    throw;
  }
  {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto key = std::make_pair(dev, dim * 16 + m.p);
    if (dim == 2 && !m.quad && !g_tab_done.count(key)) {
      tri_upload_tables(m.p, m.tab);
      DGC_CUDA(cudaGetLastError());
      g_tab_done.insert(key);
    }
  }
  // reserve the allocation-free step's array on this device now, in a call
  // that allocates anyway: the lookup loads the module that holds it (under
  // lazy module loading nothing else would before the first static step)
  static_scratch(dev, true);
  m.dev = d.release();
  m.dirty = false;
}

Mesh& checked(dgc_mesh* mesh) {
  require(mesh != nullptr, "null mesh");
  return *reinterpret_cast<Mesh*>(mesh);
}
const Mesh& checked(const dgc_mesh* mesh) {
  require(mesh != nullptr, "null mesh");
  return *reinterpret_cast<const Mesh*>(mesh);
}

// A surface-kernel tile: 16..128 edges per block (a multiple of 16), 2 or 4
// threads per edge (4: triangle meshes), at most 256 threads per block.
void check_tile(const Mesh& m, int epb, int tpe) {
  require(epb >= 16 && epb <= 128 && epb % 16 == 0, "edges per block must be 16..128, a multiple of 16");
  require(tpe == 2 || tpe == 4, "threads per edge must be 2 or 4");
  require(tpe == 2 || (m.dim == 2 && !m.quad), "4 threads per edge: triangle meshes only", DGC_ERR_UNSUPPORTED);
  require(tpe * epb <= 256, "threads per edge x edges per block must not exceed 256");
}

// The checks every device call on a mesh makes first.
void require_device_ready(const Mesh& m) {
  require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored (call dgc_color_edges first)");
  require(!m.nonaffine || m.hybrid, "general quadrilaterals need the table-driven kernels", DGC_ERR_UNSUPPORTED);
}

// The kernels' view of an uploaded mesh (d: its device arrays).
Ctx make_ctx(const Mesh& m, const DeviceMesh* d, void* stream) {
  Ctx x;
  x.dim = m.dim;
  x.quad = m.quad;
  x.hybrid = m.hybrid;
  x.p = m.p;
  x.np = m.np;
  x.M = m.M;
  x.nfpe = m.nfpe;
  x.ne = m.ne;
  x.ns = m.ns;
  x.epb = m.edges_per_block;
  x.persistent = m.persistent;
  if (m.persistent) {
    int dev = 0;
    DGC_CUDA(cudaGetDevice(&dev));
    DGC_CUDA(cudaDeviceGetAttribute(&x.sms, cudaDevAttrMultiProcessorCount, dev));
  }
  for (int c = 0; c < 3; ++c) {
    x.tile_epb[c] = m.tile_epb[c];
    x.tile_tpe[c] = m.tile_tpe[c];
  }
  x.d = d;
  x.shadow.M = m.M;
  x.shadow.np = m.np;
  x.shadow.nv = m.M * m.np;
  x.shadow.rec = (int)record_floats(m);
  x.shadow.split = true;
  x.shadow.mode_major = m.dim == 2 && !m.quad;
  x.shadow.phi0 = m.tab.phiV[0];
  x.st = static_cast<cudaStream_t>(stream);
  return x;
}

Ctx ready(Mesh& m, void* stream) {
  require_device_ready(m);
  upload(m);
  return make_ctx(m, m.dev, stream);
}

void check_ptr(const void* p, const char* what) {
  if (!p) throw Error{DGC_ERR_ARG, std::string("null device pointer: ") + what};
  if (reinterpret_cast<uintptr_t>(p) % 16) throw Error{DGC_ERR_ARG, std::string("misaligned device pointer: ") + what};
}

// ss: floats per element of an FP32 state (record or Kahan state), 0 for FP64 states
int vol(const Ctx& x, TypeCfg ty, const void* s, int ss, void* r, int64_t e0 = 0) {
  if (x.hybrid)
    return (ty == TY_D || ty == TY_MD) && e0 == 0
               ? hyb_volume(x, static_cast<const double*>(s), static_cast<double*>(r), ty == TY_MD)
               : -1;
  if (x.quad) return quad_volume(x, ty, s, ss, r, e0);
  return x.dim == 2 ? tri_volume(x, ty, s, ss, r, e0) : tet_volume(x, ty, s, ss, r, e0);
}
int surf(const Ctx& x, TypeCfg ty, SurfMode mode, int64_t b, int64_t e, const void* s, int ss, void* r, void* buf,
         const StageArgs* sa) {
  if (x.hybrid) {
    if ((ty != TY_D && ty != TY_MD) || (mode != SURF_RMW && mode != SURF_ATOMIC)) return -1;
    return hyb_surface(x, mode == SURF_ATOMIC, b, e, static_cast<const double*>(s), static_cast<double*>(r),
                       ty == TY_MD);
  }
  if (x.quad) return quad_surface(x, ty, mode, b, e, s, ss, r, buf, sa);
  return x.dim == 2 ? tri_surface(x, ty, mode, b, e, s, ss, r, buf, sa)
                    : tet_surface(x, ty, mode, b, e, s, ss, r, buf, sa);
}
// general quadrilaterals of a hybrid mesh: their mass matrices, after the colors
int mass(const Ctx& x, TypeCfg ty, void* r) {
  if (!x.hybrid) return 0;
  return ty == TY_D || ty == TY_MD ? hyb_mass(x, static_cast<double*>(r)) : -1;
}
int cfl(const Ctx& x, const double* s, double c, double* dt, float* sh) {
  if (x.hybrid) return sh ? -1 : hyb_cfl(x, s, c, dt);
  if (x.quad) return quad_cfl(x, s, c, dt, sh);
  return x.dim == 2 ? tri_cfl(x, s, c, dt, sh) : tet_cfl(x, s, c, dt, sh);
}

void count(Mesh& m, int64_t& n, int r) {
  if (r < 0) throw Error{DGC_ERR_UNSUPPORTED, "no kernel for this element type / order / precision"};
  n += r;
}

// Optional per-launch event pairs (DGC_OPT_PROFILE), recorded on the launch stream.
struct Prof {
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls, nl;
  size_t used = 0;
};

Prof* prof_of(Mesh& m) {
  if (!m.prof) m.prof = new Prof();
  return static_cast<Prof*>(m.prof);
}

void prof_free(Mesh& m) {
  if (!m.prof) return;
  Prof* P = static_cast<Prof*>(m.prof);
  for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
  delete P;
  m.prof = nullptr;
}

// launch through f(), counting its kernels; bracket it with events when profiling
template <typename F>
void run(Mesh& m, const Ctx& x, int cls, int64_t& n, F&& f) {
  Prof* P = m.profile ? prof_of(m) : nullptr;
  size_t slot = 0;
  if (P) {
    slot = P->used;
    while (P->ev.size() < slot + 2) {
      cudaEvent_t e;
      DGC_CUDA(cudaEventCreate(&e));
      P->ev.push_back(e);
    }
    P->used += 2;
    DGC_CUDA(cudaEventRecord(P->ev[slot], x.st));
  }
  const int r = f();
  if (P) {
    DGC_CUDA(cudaEventRecord(P->ev[slot + 1], x.st));
    P->cls.push_back(cls);
    P->nl.push_back(r > 0 ? r : 0);
  }
  count(m, n, r);
}

void finish(Mesh& m, int64_t launches) {
  m.last_launches = launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error{DGC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

// rhs = L(state): Algorithm 1 (volume, then the colors in order, a kernel
// boundary between colors); with fusion on closed conforming meshes the
// first color also evaluates the volume integral and stores, no pre-zeroing.
// The first color carries the volume integral (plain store) when it reaches
// every element once (closed conforming meshes), or, after the color-1
// renumbering, the elements [0, reached) it does reach; the rest get a volume
// kernel of their own.
bool first_fused(const Mesh& m) { return m.fuse && !m.hybrid && (m.perfect || m.reached >= 0); }
int64_t unreached(const Mesh& m) { return m.perfect ? m.ne : m.reached; }

int64_t launch_rhs(Mesh& m, const Ctx& x, TypeCfg ty, const void* state, int ss, void* rhs) {
  int64_t n = 0;
  const std::vector<int32_t>& off = m.color_off;
  if (m.coop && m.dim == 2 && !m.quad && (ty == TY_D || ty == TY_MD)) {
    require(!m.has_bc, "the cooperative right-hand side keeps transmissive boundaries", DGC_ERR_UNSUPPORTED);
    // every phase of Algorithm 1 in one cooperative launch
    run(m, x, DGC_K_COLOR, n, [&] {
      return tri_rhs_coop(x, ty, off.data(), m.ncolors, first_fused(m), unreached(m), state, rhs);
    });
    return n;
  }
  if (first_fused(m)) {
    run(m, x, DGC_K_FIRST, n, [&] { return surf(x, ty, SURF_FIRST, off[0], off[1], state, ss, rhs, nullptr, nullptr); });
    run(m, x, DGC_K_VOLUME, n, [&] { return vol(x, ty, state, ss, rhs, unreached(m)); });
    for (int c = 2; c <= m.ncolors; ++c)
      run(m, x, DGC_K_COLOR, n, [&] { return surf(x, ty, SURF_RMW, off[c - 1], off[c], state, ss, rhs, nullptr, nullptr); });
  } else {
    run(m, x, DGC_K_VOLUME, n, [&] { return vol(x, ty, state, ss, rhs); });
    for (int c = 1; c <= m.ncolors; ++c)
      run(m, x, DGC_K_COLOR, n, [&] { return surf(x, ty, SURF_RMW, off[c - 1], off[c], state, ss, rhs, nullptr, nullptr); });
    run(m, x, DGC_K_VOLUME, n, [&] { return mass(x, ty, rhs); });
  }
  return n;
}

// Workspace of one RK step, each part 256-byte aligned (S = FP64 state bytes,
// R = FP32 record bytes):
//   FP64:         u1 [S] (stage state), rhs [S]
//   FP32 mixed:   rec0 [R] (record of u0), recs [R] (record of the stage state),
//                 delta [S/2] (stage increment), rhs [S/2]
//   FP32 Kahan:   recs [R], delta [S/2], rhs [S/2]  (the state's first part is u0's record)
// and, last, the CFL estimates [E + 64 floats].
struct Workspace {
  double* u1 = nullptr;
  float *rec0 = nullptr, *recs = nullptr, *delta = nullptr;
  void* rhs = nullptr;
  float* est = nullptr;  // CFL estimates [E] and their minimum (so that steps on different streams never share)
  int64_t bytes = 0;
};

Workspace carve(const Mesh& m, dgc_prec prec, char* base) {
  Workspace w;
  const int64_t S = state_bytes(m), R = align256(m.ne * record_floats(m) * 4);
  int64_t o = 0;
  auto take = [&](int64_t b) {
    char* p = base ? base + o : nullptr;
    o += align256(b);
    return p;
  };
  if (prec == DGC_FP64 || m.hybrid) {  // hybrid meshes take the FP64 step in both forms
    w.u1 = reinterpret_cast<double*>(take(S));
    w.rhs = take(S);
  } else {
    if (prec == DGC_FP32_MIXED) w.rec0 = reinterpret_cast<float*>(take(R));
    w.recs = reinterpret_cast<float*>(take(R));
    w.delta = reinterpret_cast<float*>(take(S / 2));
    w.rhs = take(S / 2);
  }
  w.est = reinterpret_cast<float*>(take((m.ne + 64) * (int64_t)sizeof(float)));
  w.bytes = o;
  return w;
}

// One SSP-RK3 step.  Per stage: FIRST + COLOR... + LAST (volume integral fused
// into the first color, stage update into the last) on meshes where every
// element has one edge of each color, else VOLUME + every color + STAGE.
// launch(cls, f) issues the kernels of f() and counts them.
template <typename Launch>
void rk_step_body(const Mesh& m, const Ctx& x, dgc_prec prec, void* c, double cfl_, double* dt, const Workspace& w,
                  Launch&& launch) {
  const std::vector<int32_t>& off = m.color_off;
  const int C = m.ncolors;
  const bool fused = m.fuse && m.perfect && C >= 2;
  if (prec == DGC_FP64 || m.hybrid) {
    // (hybrid meshes in the FP32-mixed form: this FP64 step with FP32 fluxes and projections)
    const TypeCfg ty = prec == DGC_FP64 ? TY_D : TY_MD;
    double* c64 = static_cast<double*>(c);
    launch(DGC_K_CFL, [&] { return cfl(x, c64, cfl_, dt, nullptr); });
    const double A0[3] = {0.0, 0.75, 1.0 / 3.0}, B0[3] = {1.0, 0.25, 2.0 / 3.0};
    const double TF[3] = {0.0, 1.0, 0.5};  // the stages' times, in units of dt from the step's start
    for (int s = 0; s < 3; ++s) {
      Ctx xs_ = x;
      xs_.tfrac = TF[s];
      xs_.dtp = s == 0 ? nullptr : dt;  // stage 0 runs at the step's start, before dt is known
      const Ctx& x = xs_;
      double* us = s == 0 ? c64 : w.u1;
      StageArgs sa;
      sa.u0 = c64;
      sa.uout = s == 2 ? c64 : w.u1;
      sa.dt = dt;
      sa.a0 = A0[s];
      sa.b0 = B0[s];
      if (fused) {
        launch(DGC_K_FIRST, [&] { return surf(x, ty, SURF_FIRST, off[0], off[1], us, 0, w.rhs, nullptr, nullptr); });
        for (int k = 2; k < C; ++k)
          launch(DGC_K_COLOR, [&] { return surf(x, ty, SURF_RMW, off[k - 1], off[k], us, 0, w.rhs, nullptr, nullptr); });
        launch(DGC_K_LAST, [&] { return surf(x, ty, SURF_LAST, off[C - 1], off[C], us, 0, w.rhs, nullptr, &sa); });
      } else {
        int k0 = 1;
        if (first_fused(m)) {
          launch(DGC_K_FIRST, [&] { return surf(x, ty, SURF_FIRST, off[0], off[1], us, 0, w.rhs, nullptr, nullptr); });
          k0 = 2;
        }
        launch(DGC_K_VOLUME, [&] { return vol(x, ty, us, 0, w.rhs, k0 == 2 ? unreached(m) : 0); });
        for (int k = k0; k <= C; ++k)
          launch(DGC_K_COLOR, [&] { return surf(x, ty, SURF_RMW, off[k - 1], off[k], us, 0, w.rhs, nullptr, nullptr); });
        launch(DGC_K_VOLUME, [&] { return mass(x, ty, w.rhs); });
        launch(DGC_K_STAGE, [&] { return stage_update(x, false, us, w.rhs, sa); });
      }
      if (m.limit) launch(DGC_K_LIMIT, [&] { return tri_limit(x, sa.uout); });
    }
    if (m.has_bc) launch(DGC_K_LIMIT, [&] { return time_advance(x, dt); });
    return;
  }
  // FP32 forms, increment form of the step (incr_form.cuh)
  const bool kahan = prec == DGC_FP32_KAHAN;
  float* ks = kahan ? static_cast<float*>(c) : nullptr;
  const int nf = (int)record_floats(m), kf = kahan ? (int)kahan_floats(m) : 0;
  const float* rec0 = kahan ? ks : w.rec0;
  const int rec0_stride = kahan ? kf : nf;
  // mixed form on triangles with the fusions: the first color of stage 0 reads
  // the FP64 state and does pass 1 of the CFL reduction (the record of u0 and
  // the estimates); pass 2 runs between it and the next color
  const bool first_est = fused && !kahan && m.dim == 2 && !m.quad;
  if (kahan) launch(DGC_K_CFL, [&] { return tri_cfl_kahan(x, ks, cfl_, dt); });
  else if (!first_est) launch(DGC_K_CFL, [&] { return cfl(x, static_cast<double*>(c), cfl_, dt, w.rec0); });
  const double TF[3] = {0.0, 1.0, 0.5};  // the stages' times, in units of dt from the step's start
  for (int s = 0; s < 3; ++s) {
    Ctx xs_ = x;
    xs_.tfrac = TF[s];
    xs_.dtp = s == 0 ? nullptr : dt;  // stage 0 runs at the step's start, before dt is known
    const Ctx& x = xs_;
    const float* in = s == 0 ? rec0 : w.recs;
    const int ss = s == 0 ? rec0_stride : nf;
    StageArgs sa;
    sa.u0 = kahan ? nullptr : static_cast<double*>(c);
    sa.uout = kahan ? nullptr : static_cast<double*>(c);
    sa.dt = dt;
    sa.stage = s;
    sa.rec0 = rec0;
    sa.rec0_stride = rec0_stride;
    sa.rec_out = w.recs;
    sa.delta = w.delta;
    sa.kstate = ks;
    if (fused) {
      if (s == 0 && first_est) {
        launch(DGC_K_FIRST, [&] {
          return tri_first_est(x, off[0], off[1], static_cast<const double*>(c), w.rec0, static_cast<float*>(w.rhs));
        });
        launch(DGC_K_CFL, [&] { return tri_cfl_pass2(x, static_cast<const double*>(c), cfl_, dt); });
      } else {
        launch(DGC_K_FIRST,
               [&] { return surf(x, TY_MF, SURF_FIRST, off[0], off[1], in, ss, w.rhs, nullptr, nullptr); });
      }
      for (int k = 2; k < C; ++k)
        launch(DGC_K_COLOR, [&] { return surf(x, TY_MF, SURF_RMW, off[k - 1], off[k], in, ss, w.rhs, nullptr, nullptr); });
      launch(DGC_K_LAST, [&] { return surf(x, TY_MF, SURF_LAST, off[C - 1], off[C], in, ss, w.rhs, nullptr, &sa); });
    } else {
      int k0 = 1;
      if (first_fused(m)) {
        launch(DGC_K_FIRST, [&] { return surf(x, TY_MF, SURF_FIRST, off[0], off[1], in, ss, w.rhs, nullptr, nullptr); });
        k0 = 2;
      }
      launch(DGC_K_VOLUME, [&] { return vol(x, TY_MF, in, ss, w.rhs, k0 == 2 ? unreached(m) : 0); });
      for (int k = k0; k <= C; ++k)
        launch(DGC_K_COLOR, [&] { return surf(x, TY_MF, SURF_RMW, off[k - 1], off[k], in, ss, w.rhs, nullptr, nullptr); });
      launch(DGC_K_STAGE, [&] { return incr_stage_update(x, static_cast<const float*>(w.rhs), sa); });
    }
  }
  if (m.has_bc) launch(DGC_K_LIMIT, [&] { return time_advance(x, dt); });
}

}  // namespace

namespace dgc {
void device_free(Mesh& m) {
  if (!m.dev) return;
  cudaFree(m.dev->jinv);
  cudaFree(m.dev->inr);
  cudaFree(m.dev->topo);
  cudaFree(m.dev->fgeo);
  cudaFree(m.dev->slots);
  cudaFree(m.dev->perm);
  cudaFree(m.dev->xfer);
  cudaFree(m.dev->ftab);
  cudaFree(m.dev->ftabd);
  cudaFree(m.dev->ftabdf);
  cudaFree(m.dev->vtabdf);
  cudaFree(m.dev->cfl_est);
  cudaFree(m.dev->hyb_kind);
  cudaFree(m.dev->hyb_tab);
  cudaFree(m.dev->bil_slot);
  cudaFree(m.dev->bil_elem);
  cudaFree(m.dev->bil_G);
  cudaFree(m.dev->bil_Minv);
  if (m.dev->time) {  // keep the time the steps advanced to
    double t = m.time;
    if (cudaMemcpy(&t, m.dev->time, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess) m.time = t;
  }
  cudaFree(m.dev->bc);
  cudaFree(m.dev->bgeo);
  cudaFree(m.dev->time);
  cudaFree(m.dev->enb);
  cudaFree(m.dev->xf_src);
  cudaFree(m.dev->xf_kind);
  cudaFree(m.dev->xf_kids);
  cudaFree(m.dev->xf_P);
  delete m.dev;
  m.dev = nullptr;
  m.dirty = true;
}
}  // namespace dgc

extern "C" {

const char* dgc_last_error(void) { return g_err.c_str(); }

dgc_status dgc_mesh_create(int dim, int p, int64_t nv, const double* xyz, int64_t ne, const int32_t* ev,
                           const double* periodic_len, dgc_mesh** out) {
  return guarded([&] {
    require(out != nullptr, "null output pointer");
    *out = nullptr;
    *out = reinterpret_cast<dgc_mesh*>(build_mesh(dim, p, nv, xyz, ne, ev, periodic_len));
  });
}

dgc_status dgc_mesh_create_elem(dgc_elem type, int p, int64_t nv, const double* xyz, int64_t ne, const int32_t* ev,
                                const double* periodic_len, dgc_mesh** out) {
  return guarded([&] {
    require(out != nullptr, "null output pointer");
    *out = nullptr;
    require(type == DGC_TRI || type == DGC_QUAD || type == DGC_TET, "unknown element type");
    const int dim = type == DGC_TET ? 3 : 2;
    *out = reinterpret_cast<dgc_mesh*>(build_mesh(dim, p, nv, xyz, ne, ev, periodic_len, type == DGC_QUAD));
  });
}

dgc_status dgc_mesh_element(const dgc_mesh* mesh, int32_t* type, int64_t* nonaffine) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    if (type) *type = m.quad ? DGC_QUAD : m.dim == 3 ? DGC_TET : DGC_TRI;
    if (nonaffine) *nonaffine = m.nonaffine;
  });
}

static void report_colors(const Mesh& m, int32_t* n_colors, int64_t* per_color) {
  if (n_colors) *n_colors = m.ncolors;
  if (per_color) {
    for (int c = 0; c < 8; ++c) per_color[c] = 0;
    for (int c = 1; c <= m.ncolors && c <= 8; ++c) per_color[c - 1] = m.color_off[c] - m.color_off[c - 1];
  }
}

dgc_status dgc_color_edges(dgc_mesh* mesh, uint64_t seed, int64_t max_swaps, int32_t* n_colors,
                           int64_t* per_color) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    try {
      color_faces(m, seed, max_swaps);
    } catch (const Error&) {
      m.ncolors = 0;
      m.color.clear();
      m.side_old_of_new.clear();
      m.dirty = true;
      throw;
    }
    reorder(m, true, true);
    report_colors(m, n_colors, per_color);
  });
}

dgc_status dgc_color_edges_naive(dgc_mesh* mesh, int renumber, int reorder_left, int32_t* n_colors,
                                 int64_t* per_color) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    color_faces_naive(m);
    reorder(m, renumber != 0, reorder_left != 0);
    report_colors(m, n_colors, per_color);
  });
}

dgc_status dgc_reorder(dgc_mesh* mesh, int renumber, int reorder_left) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    reorder(m, renumber != 0, reorder_left != 0);
  });
}

dgc_status dgc_mesh_info(const dgc_mesh* mesh, int64_t info[10]) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(info != nullptr, "null info");
    info[0] = m.ne;
    info[1] = m.ns;
    info[2] = m.np;
    info[3] = m.M;
    info[4] = m.tab.nqf;
    info[5] = m.tab.nqv;
    info[6] = m.ncolors;
    info[7] = m.dim;
    info[8] = m.p;
    info[9] = m.perfect ? 1 : 0;
  });
}

dgc_status dgc_get_sides(const dgc_mesh* mesh, int32_t* left, int32_t* right, int8_t* qleft, int8_t* qright) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    if (left) std::copy(m.sl.begin(), m.sl.end(), left);
    if (right) std::copy(m.sr.begin(), m.sr.end(), right);
    if (qleft) std::copy(m.sql.begin(), m.sql.end(), qleft);
    if (qright) std::copy(m.sqr.begin(), m.sqr.end(), qright);
  });
}

dgc_status dgc_get_hanging(const dgc_mesh* mesh, int8_t* half) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(half != nullptr, "null argument");
    if (m.shalf.empty()) std::fill_n(half, m.ns, (int8_t)-1);
    else std::copy(m.shalf.begin(), m.shalf.end(), half);
  });
}

dgc_status dgc_get_elements(const dgc_mesh* mesh, int32_t* ev, double* xyz) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    if (ev) std::copy(m.ev.begin(), m.ev.end(), ev);
    if (xyz) std::copy(m.X.begin(), m.X.end(), xyz);
  });
}

dgc_status dgc_refine(dgc_mesh* mesh, int64_t n, const int32_t* elems) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(m.dim == 2 && !m.quad, "nonconforming refinement is implemented for triangle meshes",
            DGC_ERR_UNSUPPORTED);
    require(!m.has_bc && !m.limit, "refinement keeps transmissive boundaries and no limiter", DGC_ERR_UNSUPPORTED);
    require(!m.side_old_of_new.empty() && (m.refined || (m.ncolors == 3 && m.perfect)),
            "refine a mesh colored by dgc_color_edges with 3 colors, or one refined before");
    require(n >= 0 && (n == 0 || elems != nullptr), "bad element list");
    std::vector<uint8_t> flag(m.ne, 0);
    for (int64_t i = 0; i < n; ++i) {
      require(elems[i] >= 0 && elems[i] < m.ne, "element id out of range");
      flag[elems[i]] = 1;
    }
    refine(m, flag);
  });
}

dgc_status dgc_coarsen(dgc_mesh* mesh) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(m.refined, "the mesh is not refined");
    coarsen(m);
  });
}

dgc_status dgc_get_ordering(const dgc_mesh* mesh, int32_t* elem_new_of_old, int32_t* edge_new_of_old,
                            int8_t* edge_color, int32_t* color_offsets) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    if (elem_new_of_old) std::copy(m.elem_new_of_old.begin(), m.elem_new_of_old.end(), elem_new_of_old);
    if (edge_new_of_old) std::copy(m.side_new_of_old.begin(), m.side_new_of_old.end(), edge_new_of_old);
    if (edge_color) std::copy(m.color.begin(), m.color.end(), edge_color);
    if (color_offsets) std::copy(m.color_off.begin(), m.color_off.end(), color_offsets);
  });
}

dgc_status dgc_vol_points(const dgc_mesh* mesh, double* xyz) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(xyz != nullptr, "null output");
    vol_points(m, xyz);
  });
}

dgc_status dgc_project(const dgc_mesh* mesh, const double* vals, double* c_host) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(vals && c_host, "null array");
    project(m, vals, c_host);
  });
}

dgc_status dgc_state_size(const dgc_mesh* mesh, int64_t* bytes) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(bytes != nullptr, "null output");
    *bytes = state_bytes(m);
  });
}

static int64_t workspace_bytes(const Mesh& m, dgc_prec prec) { return carve(m, prec, nullptr).bytes; }

static void require_prec(const Mesh& m, dgc_prec prec) {
  require(prec == DGC_FP64 || prec == DGC_FP32_MIXED || prec == DGC_FP32_KAHAN, "unknown precision");
  require(!m.hybrid || prec != DGC_FP32_KAHAN, "hybrid triangle/quadrilateral meshes run in FP64 and FP32-mixed",
          DGC_ERR_UNSUPPORTED);
  require(prec != DGC_FP32_KAHAN || (m.dim == 2 && !m.quad), "the Kahan form is implemented for triangle meshes",
          DGC_ERR_UNSUPPORTED);
  require(prec == DGC_FP64 || !m.limit, "the limiter runs in FP64", DGC_ERR_UNSUPPORTED);
}

// bytes of one device state of the given precision form
static int64_t state_bytes_prec(const Mesh& m, dgc_prec prec) {
  return prec == DGC_FP32_KAHAN ? m.ne * kahan_floats(m) * (int64_t)sizeof(float) : state_bytes(m);
}

dgc_status dgc_workspace_size(const dgc_mesh* mesh, dgc_prec prec, int64_t* bytes) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(bytes != nullptr, "null output");
    require_prec(m, prec);
    *bytes = workspace_bytes(m, prec);
  });
}

dgc_status dgc_state_bytes(const dgc_mesh* mesh, dgc_prec prec, int64_t* bytes) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(bytes != nullptr, "null output");
    require_prec(m, prec);
    *bytes = state_bytes_prec(m, prec);
  });
}

// Host <-> device state copies.  The element permutation runs on the device
// (one pass over the state); a pinned (page-locked or registered) host buffer is
// copied directly, any other goes through the mesh's pinned staging buffer with
// one flat copy.
static bool host_is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

static double* xfer_of(Mesh& m) {
  if (!m.dev->xfer) m.dev->xfer = dalloc<double>(m.ne * nv_of(m));
  return m.dev->xfer;
}

dgc_status dgc_import_state(dgc_mesh* mesh, const double* c_host, double* c_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(c_host != nullptr, "null host state");
    check_ptr(c_dev, "c_dev");
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    upload(m);
    double* x = xfer_of(m);
    const int64_t S = state_bytes(m);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (host_is_pinned(c_host)) {
      DGC_CUDA(cudaMemcpyAsync(x, c_host, S, cudaMemcpyHostToDevice, st));
    } else {
      double* stg = staging_for(m);
      const int64_t n = m.ne * nv_of(m);
      parallel_for(n, [&](int64_t b, int64_t e) { std::memcpy(stg + b, c_host + b, sizeof(double) * (e - b)); });
      DGC_CUDA(cudaMemcpyAsync(x, stg, S, cudaMemcpyHostToDevice, st));
    }
    permute_blocks(st, c_dev, x, m.dev->perm, (int)nv_of(m), m.ne, true);
    DGC_CUDA(cudaGetLastError());
    DGC_CUDA(cudaStreamSynchronize(st));
  });
}

dgc_status dgc_export_state(dgc_mesh* mesh, const double* c_dev, double* c_host, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(c_host != nullptr, "null host state");
    check_ptr(c_dev, "c_dev");
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    upload(m);
    double* x = xfer_of(m);
    const int64_t S = state_bytes(m);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    permute_blocks(st, x, c_dev, m.dev->perm, (int)nv_of(m), m.ne, false);
    DGC_CUDA(cudaGetLastError());
    if (host_is_pinned(c_host)) {
      DGC_CUDA(cudaMemcpyAsync(c_host, x, S, cudaMemcpyDeviceToHost, st));
      DGC_CUDA(cudaStreamSynchronize(st));
    } else {
      double* stg = staging_for(m);
      DGC_CUDA(cudaMemcpyAsync(stg, x, S, cudaMemcpyDeviceToHost, st));
      DGC_CUDA(cudaStreamSynchronize(st));
      const int64_t n = m.ne * nv_of(m);
      parallel_for(n, [&](int64_t b, int64_t e) { std::memcpy(c_host + b, stg + b, sizeof(double) * (e - b)); });
    }
  });
}

// Stream-ordered forms for pipelining: the caller provides the device transfer
// buffer (so that copies of different steps can be in flight at once) and a
// pinned host buffer; nothing is synchronised.
dgc_status dgc_import_state_async(dgc_mesh* mesh, const double* c_host, double* c_dev, double* xfer_dev,
                                  void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(c_host != nullptr && host_is_pinned(c_host), "c_host must be pinned host memory");
    check_ptr(c_dev, "c_dev");
    check_ptr(xfer_dev, "xfer_dev");
    require(xfer_dev != c_dev, "xfer_dev and c_dev must differ");
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    upload(m);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DGC_CUDA(cudaMemcpyAsync(xfer_dev, c_host, state_bytes(m), cudaMemcpyHostToDevice, st));
    permute_blocks(st, c_dev, xfer_dev, m.dev->perm, (int)nv_of(m), m.ne, true);
    DGC_CUDA(cudaGetLastError());
  });
}

dgc_status dgc_export_state_async(dgc_mesh* mesh, const double* c_dev, double* c_host, double* xfer_dev,
                                  void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(c_host != nullptr && host_is_pinned(c_host), "c_host must be pinned host memory");
    check_ptr(c_dev, "c_dev");
    check_ptr(xfer_dev, "xfer_dev");
    require(xfer_dev != c_dev, "xfer_dev and c_dev must differ");
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    upload(m);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    permute_blocks(st, xfer_dev, c_dev, m.dev->perm, (int)nv_of(m), m.ne, false);
    DGC_CUDA(cudaGetLastError());
    DGC_CUDA(cudaMemcpyAsync(c_host, xfer_dev, state_bytes(m), cudaMemcpyDeviceToHost, st));
  });
}

// Kahan pair state of one element (triangles) from its FP64 coefficients
// [M][Np], mode-major: hi and lo of the mean phi0 c0 ([M] each), hi of mode
// j >= 1 at M (j + 1), then lo of mode j >= 1 at nf + M (j - 1); the inverse on
// export.
static void kahan_pack(const Mesh& m, const double* c, float* k) {
  const int M = m.M, np = m.np, nf = (int)record_floats(m), kf = (int)kahan_floats(m);
  const double phi0 = m.tab.phiV[0];
  std::fill(k, k + kf, 0.0f);
  for (int a = 0; a < M; ++a) {
    const double u = phi0 * c[a * np];
    const float hi = (float)u;
    k[a] = hi;
    k[M + a] = (float)(u - (double)hi);
    for (int j = 1; j < np; ++j) {
      const double v = c[a * np + j];
      const float h = (float)v;
      k[M * (j + 1) + a] = h;
      k[nf + M * (j - 1) + a] = (float)(v - (double)h);
    }
  }
}
static void kahan_unpack(const Mesh& m, const float* k, double* c) {
  const int M = m.M, np = m.np, nf = (int)record_floats(m);
  const double phi0 = m.tab.phiV[0];
  for (int a = 0; a < M; ++a) {
    c[a * np] = ((double)k[a] + (double)k[M + a]) / phi0;
    for (int j = 1; j < np; ++j) c[a * np + j] = (double)k[M * (j + 1) + a] + (double)k[nf + M * (j - 1) + a];
  }
}

dgc_status dgc_import_state_prec(dgc_mesh* mesh, dgc_prec prec, const double* c_host, void* c_dev, void* stream) {
  if (prec != DGC_FP32_KAHAN) return dgc_import_state(mesh, c_host, static_cast<double*>(c_dev), stream);
  return guarded([&] {
    Mesh& m = checked(mesh);
    require_prec(m, prec);
    require(c_host != nullptr, "null host state");
    check_ptr(c_dev, "c_dev");
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    upload(m);
    float* stg = reinterpret_cast<float*>(staging_for(m));
    const int64_t nv = nv_of(m), kf = kahan_floats(m);
    const int32_t* en = m.elem_new_of_old.data();
    parallel_for(m.ne, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) kahan_pack(m, c_host + i * nv, stg + (int64_t)en[i] * kf);
    });
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DGC_CUDA(cudaMemcpyAsync(c_dev, stg, state_bytes_prec(m, prec), cudaMemcpyHostToDevice, st));
    DGC_CUDA(cudaStreamSynchronize(st));
  });
}

dgc_status dgc_export_state_prec(dgc_mesh* mesh, dgc_prec prec, const void* c_dev, double* c_host, void* stream) {
  if (prec != DGC_FP32_KAHAN) return dgc_export_state(mesh, static_cast<const double*>(c_dev), c_host, stream);
  return guarded([&] {
    Mesh& m = checked(mesh);
    require_prec(m, prec);
    require(c_host != nullptr, "null host state");
    check_ptr(c_dev, "c_dev");
    require(m.ncolors > 0 && !m.side_old_of_new.empty(), "mesh is not colored");
    upload(m);
    float* stg = reinterpret_cast<float*>(staging_for(m));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DGC_CUDA(cudaMemcpyAsync(stg, c_dev, state_bytes_prec(m, prec), cudaMemcpyDeviceToHost, st));
    DGC_CUDA(cudaStreamSynchronize(st));
    const int64_t nv = nv_of(m), kf = kahan_floats(m);
    const int32_t* en = m.elem_new_of_old.data();
    parallel_for(m.ne, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) kahan_unpack(m, stg + (int64_t)en[i] * kf, c_host + i * nv);
    });
  });
}

dgc_status dgc_rhs(dgc_mesh* mesh, dgc_prec prec, const void* c_dev, double* rhs_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require_prec(m, prec);
    check_ptr(c_dev, "c_dev");
    check_ptr(rhs_dev, "rhs_dev");
    require(c_dev != rhs_dev, "c_dev and rhs_dev must not alias");
    Ctx x = ready(m, stream);
    x.pdl = m.pdl;
    if (prec == DGC_FP32_KAHAN) finish(m, launch_rhs(m, x, TY_KD, c_dev, (int)kahan_floats(m), rhs_dev));
    else finish(m, launch_rhs(m, x, prec == DGC_FP64 ? TY_D : TY_MD, c_dev, 0, rhs_dev));
  });
}

dgc_status dgc_set_boundary(dgc_mesh* mesh, const int8_t* kind, const int8_t* state_idx, int nstates,
                            const double* states, const double* shock, const int8_t* shock_states) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(m.dim == 2 && !m.quad, "boundary conditions: triangle meshes only", DGC_ERR_UNSUPPORTED);
    require(!m.refined, "boundary conditions: conforming meshes only", DGC_ERR_UNSUPPORTED);
    require(kind != nullptr, "null kind array");
    require(nstates >= 0 && nstates <= kBcMaxStates, "state count must be 0..8");
    require(nstates == 0 || states != nullptr, "null states");
    bool any = false, shock_used = false;
    for (int64_t s = 0; s < m.ns; ++s) {
      if (m.sr[s] >= 0) continue;
      const int k = kind[s];
      require(k >= DGC_BC_TRANSMISSIVE && k <= DGC_BC_SHOCK, "unknown boundary kind");
      if (k == DGC_BC_STATE)
        require(state_idx != nullptr && state_idx[s] >= 0 && state_idx[s] < nstates, "state index out of range");
      shock_used |= k == DGC_BC_SHOCK;
      any |= k != DGC_BC_TRANSMISSIVE;
    }
    if (shock_used)
      require(shock != nullptr && shock_states != nullptr && shock_states[0] >= 0 && shock_states[0] < nstates &&
                  shock_states[1] >= 0 && shock_states[1] < nstates,
              "shock faces need the shock and its two states");
    for (int i = 0; i < 4 * nstates; ++i) require(std::isfinite(states[i]), "states must be finite");
    m.bc_kind.assign(m.ns, 0);
    m.bc_sidx.assign(m.ns, 0);
    for (int64_t s = 0; s < m.ns; ++s)
      if (m.sr[s] < 0) {
        m.bc_kind[s] = kind[s];
        m.bc_sidx[s] = kind[s] == DGC_BC_STATE ? state_idx[s] : 0;
      }
    m.bc_states.assign(states, states + 4 * nstates);
    for (int a = 0; a < 3; ++a) m.shock[a] = shock_used ? shock[a] : 0.0;
    m.shock_st[0] = shock_used ? shock_states[0] : 0;
    m.shock_st[1] = shock_used ? shock_states[1] : 0;
    if (m.dev) {  // keep the device's time across the re-upload
      double t = m.time;
      if (m.dev->time) DGC_CUDA(cudaMemcpy(&t, m.dev->time, sizeof(double), cudaMemcpyDeviceToHost));
      m.time = t;
    }
    m.has_bc = any;
    m.dirty = true;
  });
}

dgc_status dgc_set_time(dgc_mesh* mesh, double t) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(std::isfinite(t), "time must be finite");
    m.time = t;
    if (m.dev && m.dev->time) DGC_CUDA(cudaMemcpy(m.dev->time, &t, sizeof(double), cudaMemcpyHostToDevice));
  });
}

dgc_status dgc_get_time(dgc_mesh* mesh, double* t) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(t != nullptr, "null output");
    if (m.dev && m.dev->time) DGC_CUDA(cudaMemcpy(&m.time, m.dev->time, sizeof(double), cudaMemcpyDeviceToHost));
    *t = m.time;
  });
}

dgc_status dgc_limit(dgc_mesh* mesh, dgc_prec prec, double* c_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(prec == DGC_FP64, "the limiter runs on FP64 states", DGC_ERR_UNSUPPORTED);
    require(m.dim == 2 && !m.quad && !m.refined, "the limiter: conforming triangle meshes only",
            DGC_ERR_UNSUPPORTED);
    check_ptr(c_dev, "c_dev");
    if (!m.want_enb) {
      m.want_enb = true;
      if (m.dev) device_free(m);  // the next upload adds the face neighbours
    }
    Ctx x = ready(m, stream);
    int64_t n = 0;
    run(m, x, DGC_K_LIMIT, n, [&] { return tri_limit(x, c_dev); });
    finish(m, n);
  });
}

dgc_status dgc_cfl_dt(dgc_mesh* mesh, const double* c_dev, double cfl_, double* dt_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    check_ptr(c_dev, "c_dev");
    require(dt_dev != nullptr && reinterpret_cast<uintptr_t>(dt_dev) % 8 == 0, "dt_dev must be an aligned device double");
    require(cfl_ > 0.0, "cfl must be positive");
    Ctx x = ready(m, stream);
    DGC_CUDA(cudaMemsetAsync(dt_dev, 0x7F, sizeof(double), x.st));
    int64_t n = 0;
    run(m, x, DGC_K_CFL, n, [&] { return cfl(x, c_dev, cfl_, dt_dev, nullptr); });
    finish(m, n);
  });
}

dgc_status dgc_rk_step(dgc_mesh* mesh, dgc_prec prec, void* c_dev, double cfl_, double* dt_dev,
                       void* workspace_dev, int64_t workspace_size, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require_prec(m, prec);
    check_ptr(c_dev, "c_dev");
    require(dt_dev != nullptr && reinterpret_cast<uintptr_t>(dt_dev) % 8 == 0, "dt_dev must be an aligned device double");
    require(workspace_dev != nullptr && reinterpret_cast<uintptr_t>(workspace_dev) % 256 == 0,
            "workspace must be 256-byte aligned");
    require(cfl_ > 0.0, "cfl must be positive");
    require(workspace_size >= workspace_bytes(m, prec), "workspace smaller than dgc_workspace_size()");
    Ctx x = ready(m, stream);
    const Workspace w = carve(m, prec, static_cast<char*>(workspace_dev));
    DeviceMesh dcopy = *m.dev;  // the mesh's arrays, the CFL estimates in the workspace
    dcopy.cfl_est = w.est;
    x.d = &dcopy;
    int64_t n = 0;
    DGC_CUDA(cudaMemsetAsync(dt_dev, 0x7F, sizeof(double), x.st));
    x.pdl = m.pdl;
    rk_step_body(m, x, prec, c_dev, cfl_, dt_dev, w, [&](int cls, auto&& f) { run(m, x, cls, n, f); });
    finish(m, n);
  });
}

dgc_status dgc_prolong_state(dgc_mesh* mesh, const double* c_coarse_dev, double* c_fine_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(m.refined, "mesh is not refined (dgc_refine first)");
    check_ptr(c_coarse_dev, "c_coarse_dev");
    check_ptr(c_fine_dev, "c_fine_dev");
    Ctx x = ready(m, stream);
    const int r = transfer_state(x.st, true, c_coarse_dev, c_fine_dev, m.dev->xf_src, m.dev->xf_kind, nullptr,
                                 m.dev->xf_P, m.ne, m.M, m.np);
    if (r < 0) throw Error{DGC_ERR_UNSUPPORTED, "no transfer kernel for this order"};
    finish(m, r);
  });
}

dgc_status dgc_restrict_state(dgc_mesh* mesh, const double* c_fine_dev, double* c_coarse_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(m.refined, "mesh is not refined (dgc_refine first)");
    check_ptr(c_coarse_dev, "c_coarse_dev");
    check_ptr(c_fine_dev, "c_fine_dev");
    Ctx x = ready(m, stream);
    const int r = transfer_state(x.st, false, c_fine_dev, c_coarse_dev, nullptr, nullptr, m.dev->xf_kids,
                                 m.dev->xf_P, m.base.ne, m.M, m.np);
    if (r < 0) throw Error{DGC_ERR_UNSUPPORTED, "no transfer kernel for this order"};
    finish(m, r);
  });
}

dgc_status dgc_refine_colors_device(dgc_mesh* mesh, int8_t* colors, double* ms, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(m.refined, "mesh is not refined (dgc_refine first)");
    require(colors != nullptr, "null output");
    const Mesh::Base& b = m.base;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    int8_t *bc = nullptr, *rule = nullptr, *out = nullptr;
    int32_t *bf = nullptr, *src = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto release = [&] {
      cudaFree(bc), cudaFree(rule), cudaFree(out), cudaFree(bf), cudaFree(src);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    };
    try {
      bc = dalloc<int8_t>(b.ns);
      bf = dalloc<int32_t>(b.ne * 3);
      src = dalloc<int32_t>(m.ns);
      rule = dalloc<int8_t>(m.ns);
      out = dalloc<int8_t>(m.ns);
      DGC_CUDA(cudaMemcpyAsync(bc, b.color.data(), b.ns, cudaMemcpyHostToDevice, st));
      DGC_CUDA(cudaMemcpyAsync(bf, b.face_of.data(), sizeof(int32_t) * b.ne * 3, cudaMemcpyHostToDevice, st));
      DGC_CUDA(cudaMemcpyAsync(src, b.color_src.data(), sizeof(int32_t) * m.ns, cudaMemcpyHostToDevice, st));
      DGC_CUDA(cudaMemcpyAsync(rule, b.color_rule.data(), m.ns, cudaMemcpyHostToDevice, st));
      DGC_CUDA(cudaEventCreate(&e0));
      DGC_CUDA(cudaEventCreate(&e1));
      DGC_CUDA(cudaEventRecord(e0, st));
      refine_colors(st, bc, bf, src, rule, m.ns, out);
      DGC_CUDA(cudaEventRecord(e1, st));
      DGC_CUDA(cudaMemcpyAsync(colors, out, m.ns, cudaMemcpyDeviceToHost, st));
      DGC_CUDA(cudaStreamSynchronize(st));
      DGC_CUDA(cudaGetLastError());
      if (ms) {
        float t = 0.f;
        DGC_CUDA(cudaEventElapsedTime(&t, e0, e1));
        *ms = t;
      }
    } catch (...) {
      release();
      throw;
    }
    release();
  });
}

namespace {
int tile_index(int kclass) {
  require(kclass == DGC_K_FIRST || kclass == DGC_K_COLOR || kclass == DGC_K_LAST,
          "tile class must be DGC_K_FIRST, DGC_K_COLOR or DGC_K_LAST");
  return kclass == DGC_K_FIRST ? 0 : kclass == DGC_K_COLOR ? 1 : 2;
}
}  // namespace

dgc_status dgc_set_tile(dgc_mesh* mesh, int kclass, int edges_per_block, int threads_per_edge) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    const int i = tile_index(kclass);
    check_tile(m, edges_per_block, threads_per_edge);
    m.tile_epb[i] = edges_per_block;
    m.tile_tpe[i] = threads_per_edge;
  });
}

dgc_status dgc_get_tile(const dgc_mesh* mesh, int kclass, int* edges_per_block, int* threads_per_edge) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(edges_per_block != nullptr && threads_per_edge != nullptr, "null output");
    const int i = tile_index(kclass);
    *edges_per_block = m.tile_epb[i];
    *threads_per_edge = m.tile_tpe[i];
  });
}

dgc_status dgc_autotune(dgc_mesh* mesh, dgc_prec prec, void* c_dev, double cfl_, double* dt_dev,
                        void* workspace_dev, int64_t workspace_size, int reps, void* stream, int* edges_per_block,
                        int* threads_per_edge, double* ms_per_step) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(reps > 0 && edges_per_block != nullptr && threads_per_edge != nullptr, "bad argument");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool tri32 = m.dim == 2 && !m.quad && prec != DGC_FP64;
    cudaEvent_t e0, e1;
    DGC_CUDA(cudaEventCreate(&e0));
    DGC_CUDA(cudaEventCreate(&e1));
    auto time_steps = [&]() {
      dgc_status s = dgc_rk_step(mesh, prec, c_dev, cfl_, dt_dev, workspace_dev, workspace_size, stream);
      if (s != DGC_OK) throw Error{s, g_err};
      DGC_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; ++r) {
        s = dgc_rk_step(mesh, prec, c_dev, cfl_, dt_dev, workspace_dev, workspace_size, stream);
        if (s != DGC_OK) throw Error{s, g_err};
      }
      DGC_CUDA(cudaEventRecord(e1, st));
      DGC_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      DGC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return (double)ms / reps;
    };
    // coordinate search, one kernel class at a time (last, middle, first
    // color): every tile of the candidate set with the other classes fixed
    double best = time_steps();
    const int cls[3] = {2, 1, 0};
    for (int ci : cls) {
      int be = m.tile_epb[ci], bt = m.tile_tpe[ci];
      for (int tpe : {2, 4}) {
        if (tpe == 4 && !tri32) continue;
        for (int epb : {32, 64, 128}) {
          if (tpe * epb > 256 || (epb == be && tpe == bt)) continue;
          m.tile_epb[ci] = epb;
          m.tile_tpe[ci] = tpe;
          const double t = time_steps();
          if (t < best) {
            best = t;
            be = epb;
            bt = tpe;
          }
        }
      }
      m.tile_epb[ci] = be;
      m.tile_tpe[ci] = bt;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < 3; ++i) {
      edges_per_block[i] = m.tile_epb[i];
      threads_per_edge[i] = m.tile_tpe[i];
    }
    if (ms_per_step) *ms_per_step = best;
  });
}

dgc_status dgc_rhs_atomic(dgc_mesh* mesh, dgc_prec prec, const double* c_dev, double* rhs_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(prec == DGC_FP64 || prec == DGC_FP32_MIXED, "unknown precision");
    check_ptr(c_dev, "c_dev");
    check_ptr(rhs_dev, "rhs_dev");
    Ctx x = ready(m, stream);
    x.pdl = m.pdl;
    const TypeCfg ty = prec == DGC_FP64 ? TY_D : TY_MD;
    int64_t n = 0;
    run(m, x, DGC_K_VOLUME, n, [&] { return vol(x, ty, c_dev, 0, rhs_dev); });
    run(m, x, DGC_K_ATOMIC, n, [&] { return surf(x, ty, SURF_ATOMIC, 0, m.ns, c_dev, 0, rhs_dev, nullptr, nullptr); });
    run(m, x, DGC_K_VOLUME, n, [&] { return mass(x, ty, rhs_dev); });
    finish(m, n);
  });
}

dgc_status dgc_two_pass_buffer_bytes(int64_t sides, int np, int neq, int word_bytes, int64_t* bytes) {
  return guarded([&] {
    require(bytes != nullptr && sides >= 0 && np > 0 && neq > 0 && word_bytes > 0, "bad argument");
    *bytes = 2 * (int64_t)np * neq * sides * word_bytes;
  });
}

dgc_status dgc_rhs_two_pass(dgc_mesh* mesh, dgc_prec prec, const double* c_dev, double* rhs_dev, void* buffer_dev,
                            int64_t buffer_size, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(prec == DGC_FP64 || prec == DGC_FP32_MIXED, "unknown precision");
    check_ptr(c_dev, "c_dev");
    check_ptr(rhs_dev, "rhs_dev");
    check_ptr(buffer_dev, "buffer_dev");
    require(buffer_size >= 2 * m.ns * nv_of(m) * (int64_t)sizeof(double), "buffer smaller than dgc_two_pass_buffer_bytes()");
    Ctx x = ready(m, stream);
    x.pdl = m.pdl;
    const TypeCfg ty = prec == DGC_FP64 ? TY_D : TY_MD;
    int64_t n = 0;
    run(m, x, DGC_K_VOLUME, n, [&] { return vol(x, ty, c_dev, 0, rhs_dev); });
    run(m, x, DGC_K_BUFFER, n, [&] { return surf(x, ty, SURF_BUFFER, 0, m.ns, c_dev, 0, rhs_dev, buffer_dev, nullptr); });
    run(m, x, DGC_K_GATHER, n, [&] { return gather_two_pass(x, false, rhs_dev, buffer_dev); });
    finish(m, n);
  });
}

dgc_status dgc_set_option(dgc_mesh* mesh, dgc_option opt, int64_t value) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    switch (opt) {
      case DGC_OPT_FUSE:
        m.fuse = value != 0;
        break;
      case DGC_OPT_EDGES_PER_BLOCK:
        for (int c = 0; c < 3; ++c) check_tile(m, (int)value, m.tile_tpe[c]);
        m.edges_per_block = (int)value;
        for (int c = 0; c < 3; ++c) m.tile_epb[c] = (int)value;
        break;
      case DGC_OPT_THREADS_PER_EDGE:
        for (int c = 0; c < 3; ++c) check_tile(m, m.tile_epb[c], (int)value);
        for (int c = 0; c < 3; ++c) m.tile_tpe[c] = (int)value;
        break;
      case DGC_OPT_PROFILE:
        m.profile = value != 0;
        break;
      case DGC_OPT_PDL:
        m.pdl = value != 0;
        break;
      case DGC_OPT_PERSISTENT:
        require(value == 0 || (m.dim == 2 && !m.quad), "persistent surface kernels: triangle meshes only",
                DGC_ERR_UNSUPPORTED);
        m.persistent = value != 0;
        break;
      case DGC_OPT_LIMITER:
        require(value == 0 || (m.dim == 2 && !m.quad && !m.refined),
                "the limiter: conforming triangle meshes only", DGC_ERR_UNSUPPORTED);
        m.limit = value != 0;
        if (m.limit && !m.want_enb) {
          m.want_enb = true;
          if (m.dev) device_free(m);  // the next upload adds the face neighbours
        }
        break;
      case DGC_OPT_COOPERATIVE:
        require(value == 0 || (m.dim == 2 && !m.quad), "cooperative right-hand side: triangle meshes only",
                DGC_ERR_UNSUPPORTED);
        m.coop = value != 0;
        break;
      default:
        throw Error{DGC_ERR_ARG, "unknown option"};
    }
  });
}

dgc_status dgc_profile_collect(dgc_mesh* mesh, double* ms, int64_t* launches) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require(ms && launches, "null output");
    if (!m.prof) return;
    Prof* P = static_cast<Prof*>(m.prof);
    for (size_t i = 0; i < P->cls.size(); ++i) {
      DGC_CUDA(cudaEventSynchronize(P->ev[2 * i + 1]));
      float t = 0.f;
      DGC_CUDA(cudaEventElapsedTime(&t, P->ev[2 * i], P->ev[2 * i + 1]));
      ms[P->cls[i]] += t;
      launches[P->cls[i]] += P->nl[i];
    }
    P->cls.clear();
    P->nl.clear();
    P->used = 0;
  });
}

dgc_status dgc_last_launch_count(const dgc_mesh* mesh, int64_t* launches) {
  return guarded([&] {
    const Mesh& m = checked(mesh);
    require(launches != nullptr, "null output");
    *launches = m.last_launches;
  });
}

void dgc_destroy(dgc_mesh* mesh) {
  if (!mesh) return;
  Mesh* m = reinterpret_cast<Mesh*>(mesh);
  device_free(*m);
  staging_free(*m);
  prof_free(*m);
  delete m;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free RK step.  Its workspace (stage state, FP32 record, rhs) and
// the CFL estimates live in one file-scope device array, so the call needs no
// buffer from the caller and allocates nothing.  The array's device memory is
// reserved when this file's module is loaded on a device, which the first mesh
// upload on that device forces (upload() looks the address up); every GPU the
// library has uploaded a mesh to holds it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kStaticScratchBytes = int64_t(1) << 24;  // 16 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// In host code the array's name is only a host-side stand-in, so its address
// is looked up with the device current.  Every mesh upload (load) looks it up
// again, which loads the module on a new context, and caches it; the step only
// reads the cache.  A context reset (cudaDeviceReset) frees the array with
// every other device buffer the library holds: meshes must be destroyed before
// one and re-created (uploaded again, refreshing the address) after.
void* static_scratch(int dev, bool load) {
  if (dev < 0 || dev >= kMaxDevices) throw Error{DGC_ERR_UNSUPPORTED, "device index out of range"};
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (load) {
    void* p = nullptr;
    DGC_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[dev] = p;
  } else if (!g_static_addr[dev]) {
    throw Error{DGC_ERR_ARG, "the static array is not reserved on this device: upload a mesh first"};
  }
  return g_static_addr[dev];
}

}  // namespace

extern "C" dgc_status dgc_rk_step_static(dgc_mesh* mesh, dgc_prec prec, void* c_dev, double cfl_,
                                         double* dt_dev, void* stream) {
  return guarded([&] {
    Mesh& m = checked(mesh);
    require_prec(m, prec);
    check_ptr(c_dev, "c_dev");
    require(dt_dev != nullptr && reinterpret_cast<uintptr_t>(dt_dev) % 8 == 0, "dt_dev must be an aligned device double");
    require(cfl_ > 0.0, "cfl must be positive");
    require_device_ready(m);
    const int64_t ws = workspace_bytes(m, prec);
    if (ws > kStaticScratchBytes)
      throw Error{DGC_ERR_ARG, "mesh too large for dgc_rk_step_static: needs " + std::to_string(ws) +
                                   " bytes of scratch, the static array holds " + std::to_string(kStaticScratchBytes)};
    int dev = -1;
    DGC_CUDA(cudaGetDevice(&dev));
    // uploading the mesh would allocate: an earlier device call must have done it
    require(m.dev != nullptr && !m.dirty && m.dev->device == dev,
            "mesh not on this device yet: make one device call on it first (e.g. dgc_cfl_dt)");
    char* base = static_cast<char*>(static_scratch(dev, false));  // reserved by the upload
    const Workspace w = carve(m, prec, base);
    DeviceMesh dcopy = *m.dev;  // the same mesh arrays, CFL estimates in the static array
    dcopy.cfl_est = w.est;
    Ctx x = make_ctx(m, &dcopy, stream);
    int64_t n = 0;
    DGC_CUDA(cudaMemsetAsync(dt_dev, 0x7F, sizeof(double), x.st));
    x.pdl = m.pdl;
    rk_step_body(m, x, prec, c_dev, cfl_, dt_dev, w, [&](int, auto&& f) { count(m, n, f()); });
    finish(m, n);
  });
}

// ---------------------------------------------------------------------------
// Batches of independent triangle meshes (uneven size and order): one
// persistent launch per kernel class and RK stage covers every mesh, the whole
// step optionally replayed from a CUDA graph.
// ---------------------------------------------------------------------------
struct dgc_batch {
  std::vector<Mesh*> meshes;
  int epb = 64;                    // DGC_OPT_EDGES_PER_BLOCK (all classes)
  int tepb[3] = {64, 64, 64};      // tile of the first, middle, last color: edges per block
  int ttpe[3] = {2, 2, 2};         // and threads per edge (4: FP32-mixed form only)
  bool use_graph = true;
  int device = -1;
  // device tables, rebuilt when the call's buffers or the tile size change
  BatchMeshDev* dmeshes = nullptr;
  BatchTile* dtiles = nullptr;  // colors 1..C then elements
  int tile_off[8] = {0};        // tile ranges: color c in [tile_off[c-1], tile_off[c]), elements last
  int ncolors = 0;
  std::vector<double*> key_c;
  double* key_dt = nullptr;
  void* key_ws = nullptr;
  int key_prec = -1, key_epb[3] = {-1, -1, -1}, key_tpe[3] = {-1, -1, -1};
  cudaGraphExec_t exec = nullptr;
  double graph_cfl = 0.0;
  // the step is captured on this library-owned stream (capture is not allowed
  // on the legacy default stream a caller may pass) and launched on the caller's
  cudaStream_t capture_stream = nullptr;
  int64_t launches = 0;
  // DGC_OPT_PROFILE: an event pair around every launch (the step then runs
  // without its graph), per kernel class, for dgc_batch_profile_collect
  bool profile = false;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pcls;
  size_t pused = 0;
};

namespace {

void batch_release(dgc_batch& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  b.exec = nullptr;
  if (b.capture_stream) cudaStreamDestroy(b.capture_stream);
  b.capture_stream = nullptr;
  cudaFree(b.dmeshes);
  cudaFree(b.dtiles);
  b.dmeshes = nullptr;
  b.dtiles = nullptr;
  b.key_prec = -1;
}

int64_t batch_ws_bytes(const dgc_batch& b, dgc_prec prec) {
  int64_t t = 0;
  for (const Mesh* m : b.meshes) t += workspace_bytes(*m, prec);
  return t;
}

// tile class of color c of C: first, middle, last
int batch_class(int c, int C) { return c == 1 ? 0 : c == C ? 2 : 1; }

// descriptors and tiles for this call's buffers (host work + one synchronous upload)
void batch_prepare(dgc_batch& b, dgc_prec prec, double* const* c_devs, double* dt_devs, void* ws) {
  const int n = (int)b.meshes.size();
  bool same = b.dmeshes && b.key_prec == (int)prec && b.key_dt == dt_devs && b.key_ws == ws &&
              std::equal(b.tepb, b.tepb + 3, b.key_epb) && std::equal(b.ttpe, b.ttpe + 3, b.key_tpe);
  for (int i = 0; same && i < n; ++i) same = b.key_c[i] == c_devs[i];
  if (same) return;
  batch_release(b);
  std::vector<BatchMeshDev> hm(n);
  char* w = static_cast<char*>(ws);
  for (int i = 0; i < n; ++i) {
    Mesh& m = *b.meshes[i];
    upload(m);
    const Workspace part = carve(m, prec, w);
    BatchMeshDev& d = hm[i];
    d.p = m.p;
    d.ne = m.ne;
    d.topo = m.dev->topo;
    d.fgeo = m.dev->fgeo;
    d.jinv = m.dev->jinv;
    d.inr = m.dev->inr;
    d.est = part.est;
    d.c = c_devs[i];
    d.dt = dt_devs + i;
    d.u1 = part.u1;
    d.rec0 = part.rec0;
    d.recs = part.recs;
    d.delta = part.delta;
    d.rhs = part.rhs;
    w += part.bytes;
  }
  // tiles: every color's edges, then the elements; heavier orders first
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b.meshes[a]->p > b.meshes[c]->p; });
  std::vector<BatchTile> tiles;
  b.ncolors = b.meshes[0]->ncolors;
  b.tile_off[0] = 0;
  for (int c = 1; c <= b.ncolors; ++c) {
    const int epb = b.tepb[batch_class(c, b.ncolors)];
    for (int i : order) {
      const Mesh& m = *b.meshes[i];
      for (int64_t s = m.color_off[c - 1]; s < m.color_off[c]; s += epb)
        tiles.push_back({i, m.p, s, std::min<int64_t>(s + epb, m.color_off[c])});
    }
    b.tile_off[c] = (int)tiles.size();
  }
  for (int i : order) {
    const Mesh& m = *b.meshes[i];
    for (int64_t e = 0; e < m.ne; e += 128) tiles.push_back({i, m.p, e, std::min<int64_t>(e + 128, m.ne)});
  }
  b.tile_off[b.ncolors + 1] = (int)tiles.size();
  b.dmeshes = dalloc<BatchMeshDev>(n);
  b.dtiles = dalloc<BatchTile>((int64_t)tiles.size());
  DGC_CUDA(cudaMemcpy(b.dmeshes, hm.data(), sizeof(BatchMeshDev) * n, cudaMemcpyHostToDevice));
  DGC_CUDA(cudaMemcpy(b.dtiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice));
  b.key_c.assign(c_devs, c_devs + n);
  b.key_dt = dt_devs;
  b.key_ws = ws;
  b.key_prec = (int)prec;
  std::copy(b.tepb, b.tepb + 3, b.key_epb);
  std::copy(b.ttpe, b.ttpe + 3, b.key_tpe);
}

// with DGC_OPT_PROFILE, f()'s launches between an event pair of class cls
template <typename F>
int batch_run(dgc_batch& b, cudaStream_t st, int cls, F&& f) {
  if (!b.profile) return f();
  while (b.pev.size() < b.pused + 2) {
    cudaEvent_t e;
    DGC_CUDA(cudaEventCreate(&e));
    b.pev.push_back(e);
  }
  DGC_CUDA(cudaEventRecord(b.pev[b.pused], st));
  const int r = f();
  DGC_CUDA(cudaEventRecord(b.pev[b.pused + 1], st));
  b.pused += 2;
  b.pcls.push_back(cls);
  return r;
}

// the launches of one step: reset, CFL (2), then per stage the three colors
int64_t batch_enqueue(dgc_batch& b, dgc_prec prec, double cfl_, cudaStream_t st) {
  const bool mixed = prec == DGC_FP32_MIXED;
  const int n = (int)b.meshes.size(), C = b.ncolors;
  int64_t launches = batch_run(b, st, DGC_K_CFL, [&] { return batch_init(st, b.dmeshes, n); });
  const BatchTile* et = b.dtiles + b.tile_off[C];
  launches += batch_run(b, st, DGC_K_CFL, [&] {
    return batch_cfl(st, b.dmeshes, et, b.tile_off[C + 1] - b.tile_off[C], cfl_, mixed);
  });
  const double A0[3] = {0.0, 0.75, 1.0 / 3.0}, B0[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int s = 0; s < 3; ++s)
    for (int c = 1; c <= C; ++c) {
      const SurfMode mode = c == 1 ? SURF_FIRST : (c == C ? SURF_LAST : SURF_RMW);
      const int k = batch_class(c, C), tpe = mixed ? b.ttpe[k] : 2;
      const int cls = k == 0 ? DGC_K_FIRST : k == 2 ? DGC_K_LAST : DGC_K_COLOR;
      const int r = batch_run(b, st, cls, [&] {
        return batch_surf(st, b.dmeshes, b.dtiles + b.tile_off[c - 1], b.tile_off[c] - b.tile_off[c - 1], s, A0[s],
                          B0[s], mode, mixed, tpe * b.tepb[k], tpe);
      });
      if (r < 0) throw Error{DGC_ERR_UNSUPPORTED, "no batched kernel for this configuration"};
      launches += r;
    }
  return launches;
}

dgc_batch& checked_batch(dgc_batch* b) {
  require(b != nullptr, "null batch");
  return *b;
}

}  // namespace

extern "C" {

dgc_status dgc_batch_create(int n, dgc_mesh* const* meshes, dgc_batch** out) {
  return guarded([&] {
    require(out != nullptr && meshes != nullptr && n > 0, "need a positive number of meshes");
    *out = nullptr;
    auto b = std::make_unique<dgc_batch>();
    for (int i = 0; i < n; ++i) {
      Mesh& m = checked(meshes[i]);
      require(m.dim == 2 && !m.quad, "batches hold triangle meshes");
      require(!m.has_bc && !m.limit, "batched meshes keep transmissive boundaries and no limiter",
              DGC_ERR_UNSUPPORTED);
      require(m.ncolors == 3 && m.perfect && !m.side_old_of_new.empty(),
              "batched meshes must be colored with 3 colors, every element with one edge of each color");
      b->meshes.push_back(&m);
    }
    *out = b.release();
  });
}

dgc_status dgc_batch_workspace_size(const dgc_batch* batch, dgc_prec prec, int64_t* bytes) {
  return guarded([&] {
    require(batch != nullptr && bytes != nullptr, "null argument");
    require(prec == DGC_FP64 || prec == DGC_FP32_MIXED, "unknown precision");
    *bytes = batch_ws_bytes(*batch, prec);
  });
}

dgc_status dgc_batch_set_option(dgc_batch* batch, dgc_option opt, int64_t value) {
  return guarded([&] {
    dgc_batch& b = checked_batch(batch);
    if (opt == DGC_OPT_EDGES_PER_BLOCK) {
      require(value >= 16 && value <= 128 && value % 16 == 0, "edges per block must be 16..128, a multiple of 16");
      for (int k = 0; k < 3; ++k) require(b.ttpe[k] * value <= 256, "threads per edge x edges per block > 256");
      b.epb = (int)value;
      for (int k = 0; k < 3; ++k) b.tepb[k] = (int)value;
      if (b.exec) cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
    } else if (opt == DGC_OPT_THREADS_PER_EDGE) {
      require(value == 2 || value == 4, "threads per edge must be 2 or 4");
      for (int k = 0; k < 3; ++k) require(value * b.tepb[k] <= 256, "threads per edge x edges per block > 256");
      for (int k = 0; k < 3; ++k) b.ttpe[k] = (int)value;
      if (b.exec) cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
    } else if (opt == DGC_OPT_PROFILE) {
      b.profile = value != 0;
    } else if (opt == DGC_OPT_GRAPH) {
      b.use_graph = value != 0;
      if (b.exec) cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
    } else {
      throw Error{DGC_ERR_ARG, "option not available for batches"};
    }
  });
}

dgc_status dgc_batch_rk_step(dgc_batch* batch, dgc_prec prec, double* const* c_devs, double cfl_, double* dt_devs,
                             void* workspace_dev, int64_t workspace_size, void* stream) {
  return guarded([&] {
    dgc_batch& b = checked_batch(batch);
    require(prec == DGC_FP64 || prec == DGC_FP32_MIXED, "unknown precision");
    require(c_devs != nullptr, "null state array");
    for (size_t i = 0; i < b.meshes.size(); ++i) check_ptr(c_devs[i], "c_devs[i]");
    require(dt_devs != nullptr && reinterpret_cast<uintptr_t>(dt_devs) % 8 == 0, "dt_devs must be an aligned device array");
    require(workspace_dev != nullptr && reinterpret_cast<uintptr_t>(workspace_dev) % 256 == 0,
            "workspace must be 256-byte aligned");
    require(workspace_size >= batch_ws_bytes(b, prec), "workspace smaller than dgc_batch_workspace_size()");
    require(cfl_ > 0.0, "cfl must be positive");
    int dev = -1;
    DGC_CUDA(cudaGetDevice(&dev));
    require(b.device < 0 || b.device == dev, "batch was used on another device");
    b.device = dev;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    batch_prepare(b, prec, c_devs, dt_devs, workspace_dev);
    if (!b.use_graph || b.profile) {
      b.launches = batch_enqueue(b, prec, cfl_, st);
    } else {
      if (!b.exec || b.graph_cfl != cfl_) {
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        cudaGraph_t g = nullptr;
        if (!b.capture_stream) DGC_CUDA(cudaStreamCreateWithFlags(&b.capture_stream, cudaStreamNonBlocking));
        const cudaStream_t cs = b.capture_stream;
        DGC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int64_t n = 0;
        try {
          n = batch_enqueue(b, prec, cfl_, cs);
        } catch (...) {
          cudaStreamEndCapture(cs, &g);
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          throw;
        }
        DGC_CUDA(cudaStreamEndCapture(cs, &g));
        cudaError_t e = cudaGraphInstantiate(&b.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) throw Error{DGC_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)};
        b.graph_cfl = cfl_;
        b.launches = n;
      }
      DGC_CUDA(cudaGraphLaunch(b.exec, st));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error{DGC_ERR_CUDA, std::string("batched step: ") + cudaGetErrorString(e)};
  });
}

dgc_status dgc_batch_autotune(dgc_batch* batch, dgc_prec prec, double* const* c_devs, double cfl_, double* dt_devs,
                              void* workspace_dev, int64_t workspace_size, int reps, void* stream,
                              int* edges_per_block, int* threads_per_edge, double* ms_per_step) {
  return guarded([&] {
    dgc_batch& b = checked_batch(batch);
    require(reps > 0 && edges_per_block != nullptr && threads_per_edge != nullptr, "bad argument");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    DGC_CUDA(cudaEventCreate(&e0));
    DGC_CUDA(cudaEventCreate(&e1));
    auto time_steps = [&]() {
      if (b.exec) cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
      dgc_status s = dgc_batch_rk_step(batch, prec, c_devs, cfl_, dt_devs, workspace_dev, workspace_size, stream);
      if (s != DGC_OK) throw Error{s, g_err};
      DGC_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; ++r) {
        s = dgc_batch_rk_step(batch, prec, c_devs, cfl_, dt_devs, workspace_dev, workspace_size, stream);
        if (s != DGC_OK) throw Error{s, g_err};
      }
      DGC_CUDA(cudaEventRecord(e1, st));
      DGC_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      DGC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return (double)ms / reps;
    };
    // coordinate search over the last, middle and first colors' tiles: edges
    // per block 16..128 x threads per edge 2 or 4 (FP32-mixed form)
    double best = time_steps();
    for (int k : {2, 1, 0}) {
      int be = b.tepb[k], bt = b.ttpe[k];
      for (int tpe : {2, 4}) {
        if (tpe == 4 && prec != DGC_FP32_MIXED) continue;
        for (int epb : {16, 32, 64, 128}) {
          if (tpe * epb > 256 || (epb == be && tpe == bt)) continue;
          b.tepb[k] = epb;
          b.ttpe[k] = tpe;
          const double t = time_steps();
          if (t < best) {
            best = t;
            be = epb;
            bt = tpe;
          }
        }
      }
      b.tepb[k] = be;
      b.ttpe[k] = bt;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b.exec) cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
    for (int k = 0; k < 3; ++k) {
      edges_per_block[k] = b.tepb[k];
      threads_per_edge[k] = b.ttpe[k];
    }
    if (ms_per_step) *ms_per_step = best;
  });
}

dgc_status dgc_batch_set_tile(dgc_batch* batch, int kclass, int edges_per_block, int threads_per_edge) {
  return guarded([&] {
    dgc_batch& b = checked_batch(batch);
    const int k = tile_index(kclass);
    require(edges_per_block >= 16 && edges_per_block <= 128 && edges_per_block % 16 == 0,
            "edges per block must be 16..128, a multiple of 16");
    require(threads_per_edge == 2 || threads_per_edge == 4, "threads per edge must be 2 or 4");
    require(threads_per_edge * edges_per_block <= 256, "threads per edge x edges per block must not exceed 256");
    b.tepb[k] = edges_per_block;
    b.ttpe[k] = threads_per_edge;
    if (b.exec) cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
  });
}

dgc_status dgc_batch_profile_collect(dgc_batch* batch, double* ms, int64_t* launches) {
  return guarded([&] {
    dgc_batch& b = checked_batch(batch);
    require(ms != nullptr && launches != nullptr, "null output");
    for (size_t i = 0; i < b.pcls.size(); ++i) {
      DGC_CUDA(cudaEventSynchronize(b.pev[2 * i + 1]));
      float t = 0.f;
      DGC_CUDA(cudaEventElapsedTime(&t, b.pev[2 * i], b.pev[2 * i + 1]));
      ms[b.pcls[i]] += t;
      launches[b.pcls[i]] += 1;
    }
    b.pcls.clear();
    b.pused = 0;
  });
}

dgc_status dgc_batch_launch_count(const dgc_batch* batch, int64_t* launches) {
  return guarded([&] {
    require(batch != nullptr && launches != nullptr, "null argument");
    *launches = batch->launches;
  });
}

void dgc_batch_destroy(dgc_batch* batch) {
  if (!batch) return;
  batch_release(*batch);
  for (cudaEvent_t e : batch->pev) cudaEventDestroy(e);
  delete batch;
}

}  // extern "C"
