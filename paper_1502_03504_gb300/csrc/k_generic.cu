// Plain sweeps on the generic kernels (trapezoid tiles, direct, column
// march), their support checks and shared-memory sizing; multi-stage forms
// are routed to k_generic_rk.cu.
#include "generic_kernels.cuh"

namespace lope {

size_t trap_smem_bytes(int dtype, int nf, int tile_x, int tile_y, int halo, int stages) {
  const size_t csz = dtype == kF64 ? 8 : 4;
  const size_t nbuf = stages >= 2 ? 3 : 2;
  return nbuf * size_t(nf) * size_t(tile_x + 2 * halo) * size_t(tile_y + 2 * halo) * csz;
}

// Whether any side of the grid reads an external halo (decomposed slabs);
// only the TMA and direct kernels read those.
bool has_external(const Geom& g) {
  for (int ax = 0; ax < 3; ++ax)
    for (int sd = 0; sd < 2; ++sd)
      if (g.bc[ax][sd] == kExternal) return true;
  return false;
}

bool trap2d_supported(const StepArgs& a) {
  if (a.g.ndim != 2 || a.adjoint || has_external(a.g)) return false;
  const int TX = a.tile_x > 0 ? a.tile_x : 64, TY = a.tile_y > 0 ? a.tile_y : 32;
  if (TX < 8 || TY < 1 || TX > 256 || TY > 256 || a.ksteps < 1 || a.ksteps > 8) return false;
  const int stages = std::max(1, a.s.stages);
  return trap_smem_bytes(a.g.dtype, a.g.nf, TX, TY, a.s.radius * a.ksteps * stages, stages) <=
         200 * 1024;
}

bool direct_supported(const StepArgs& a) { return a.ksteps == 1; }

bool march_supported(const StepArgs& a) {
  int blocks = 0, zchunk = 0;
  // Run-time compiled functions take the copied-plane z-march: one-field star
  // functions with FP32 / FP64 storage, plain sweeps only.
  const bool user_ok = a.s.kind != kUser || (a.s.star && a.g.nf == 1 && a.g.dtype != kBF16 &&
                                             a.s.stages == 1 && a.stage < 2);
  return a.g.ndim == 3 && !a.adjoint && user_ok && a.ksteps == 1 && !has_external(a.g) &&
         march_geometry(a.g, &blocks, &zchunk);
}

cudaError_t launch_trap2d(const StepArgs& a) {
  if (a.s.kind == kUser) return jit_launch(a, kPathTrap);
  if (a.s.stages >= 2) return launch_generic_rk(a, kGenTrap, nullptr);
  return dispatch_generic<false>(a, kGenTrap, nullptr);
}
cudaError_t launch_direct(const StepArgs& a, int* blocks) {
  if (a.s.kind == kUser) {
    if (blocks) *blocks = direct_grid(a.g);
    return jit_launch(a, kPathDirect);
  }
  if (a.stage >= 2) return launch_generic_rk(a, kGenDirect, blocks);
  return dispatch_generic<false>(a, kGenDirect, blocks);
}
cudaError_t launch_march(const StepArgs& a) {
  if (a.s.kind == kUser) return jit_launch(a, kPathMarch);
  if (a.stage >= 2) return launch_generic_rk(a, kGenMarch, nullptr);
  return dispatch_generic<false>(a, kGenMarch, nullptr);
}
int direct_blocks(const StepArgs& a) { return direct_grid(a.g); }

}  // namespace lope
