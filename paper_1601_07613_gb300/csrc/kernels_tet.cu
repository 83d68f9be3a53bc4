// Tetrahedral kernels (4-face coloring, Sec. 3): not built yet; the entry
// points report DGC_ERR_UNSUPPORTED through a negative launch count.
#include "device.cuh"

namespace dgc {
void tet_upload_tables(int, const RefTables&, DeviceMesh&) {}
int tet_volume(const Ctx&, TypeCfg, const void*, void*) { return -1; }
int tet_surface(const Ctx&, TypeCfg, SurfMode, int64_t, int64_t, const void*, void*, void*, const StageArgs*) {
  return -1;
}
int tet_cfl(const Ctx&, const double*, double, double*, float*) { return -1; }
}  // namespace dgc
