// kernels_f32.cu - FP32-factor instantiations of the fused spMTTKRP + remap kernels.
#include "mttkrp_direct.cuh"
#include "mttkrp_kernel.cuh"

namespace spm {

static int launch_direct_float(const MttkrpArgs& a, const LaneCfg& c, cudaStream_t s) {
  if (c.vec) {
    switch (a.nmodes) {
      case 3:
        if (a.es == 16) return launch_direct<3, float, 4, 1, 4>(a, c.L, s);
        return launch_direct<0, float, 4, 1, 2>(a, c.L, s);
      case 4: return launch_direct<4, float, 4, 1, 4>(a, c.L, s);
      case 5: return launch_direct<5, float, 4, 1, 4>(a, c.L, s);
      case 6: return launch_direct<6, float, 4, 1, 4>(a, c.L, s);
      default: return launch_direct<0, float, 4, 1, 2>(a, c.L, s);
    }
  }
  switch (c.RC) {
    case 1: return launch_direct<0, float, 1, 1, 2>(a, c.L, s);
    case 2: return launch_direct<0, float, 1, 2, 2>(a, c.L, s);
    case 4: return launch_direct<0, float, 1, 4, 2>(a, c.L, s);
    default: return launch_direct<0, float, 1, 8, 2>(a, c.L, s);
  }
}

int launch_mttkrp_f32(const MttkrpArgs& a, const LaneCfg& c, cudaStream_t s) {
  if (a.loss_part) {  // fused CP-loss pass (3 modes, 16- or 32-byte nonzeros, vector lanes)
    if (!(c.vec && a.nmodes == 3 && (a.es == 32 || a.es == 16)))
      return fail(SPM_ERR_UNSUPPORTED,
                  "fused CP-loss pass: 3 modes, 16- or 32-byte nonzeros only");
    if (a.es == 16) {
      switch (a.mode) {
        case 0: return launch_warp_kernel<3, float, 4, 1, 4, 0, 16, true>(a, c.L, s);
        case 1: return launch_warp_kernel<3, float, 4, 1, 4, 1, 16, true>(a, c.L, s);
        default: return launch_warp_kernel<3, float, 4, 1, 4, 2, 16, true>(a, c.L, s);
      }
    }
    switch (a.mode) {
      case 0: return launch_warp_kernel<3, float, 4, 1, 4, 0, 32, true>(a, c.L, s);
      case 1: return launch_warp_kernel<3, float, 4, 1, 4, 1, 32, true>(a, c.L, s);
      default: return launch_warp_kernel<3, float, 4, 1, 4, 2, 32, true>(a, c.L, s);
    }
  }
  if (a.variant == 3) {  // form 3: one remap warp per CTA (the dispatcher checked the layout)
    switch (a.mode) {
      case 0: return launch_warp_kernel<3, float, 4, 1, 8, 0, 32, false, true>(a, c.L, s);
      case 1: return launch_warp_kernel<3, float, 4, 1, 8, 1, 32, false, true>(a, c.L, s);
      default: return launch_warp_kernel<3, float, 4, 1, 8, 2, 32, false, true>(a, c.L, s);
    }
  }
  if (a.variant == 1) return launch_direct_float(a, c, s);
  if (c.vec) {
    switch (a.nmodes) {
      case 3:
        if (a.es == 32 && a.unroll == 4) {  // 32-byte nonzeros, 4 in flight, 3 CTAs/SM
          switch (a.mode) {
            case 0: return launch_warp_kernel<3, float, 4, 1, 4, 0, 32>(a, c.L, s);
            case 1: return launch_warp_kernel<3, float, 4, 1, 4, 1, 32>(a, c.L, s);
            default: return launch_warp_kernel<3, float, 4, 1, 4, 2, 32>(a, c.L, s);
          }
        }
        if (a.es == 32) {  // elements padded to a full 32-byte sector
          switch (a.mode) {
            case 0: return launch_warp_kernel<3, float, 4, 1, 8, 0, 32>(a, c.L, s);
            case 1: return launch_warp_kernel<3, float, 4, 1, 8, 1, 32>(a, c.L, s);
            default: return launch_warp_kernel<3, float, 4, 1, 8, 2, 32>(a, c.L, s);
          }
        }
        if (a.unroll == 4) {
          switch (a.mode) {
            case 0: return launch_warp_kernel<3, float, 4, 1, 4, 0>(a, c.L, s);
            case 1: return launch_warp_kernel<3, float, 4, 1, 4, 1>(a, c.L, s);
            default: return launch_warp_kernel<3, float, 4, 1, 4, 2>(a, c.L, s);
          }
        }
        switch (a.mode) {
          case 0: return launch_warp_kernel<3, float, 4, 1, 8, 0>(a, c.L, s);
          case 1: return launch_warp_kernel<3, float, 4, 1, 8, 1>(a, c.L, s);
          default: return launch_warp_kernel<3, float, 4, 1, 8, 2>(a, c.L, s);
        }
      case 4: return launch_warp_kernel<4, float, 4, 1, 4>(a, c.L, s);
      case 5: return launch_warp_kernel<5, float, 4, 1, 4>(a, c.L, s);
      case 6: return launch_warp_kernel<6, float, 4, 1, 4>(a, c.L, s);
      default: return launch_warp_kernel<0, float, 4, 1, 4>(a, c.L, s);
    }
  }
  switch (c.RC) {
    case 1: return launch_warp_kernel<0, float, 1, 1, 4>(a, c.L, s);
    case 2: return launch_warp_kernel<0, float, 1, 2, 4>(a, c.L, s);
    case 4: return launch_warp_kernel<0, float, 1, 4, 2>(a, c.L, s);
    default: return launch_warp_kernel<0, float, 1, 8, 1>(a, c.L, s);
  }
}

}  // namespace spm
