// kernels_tile.cu - instantiations of the tile form of the fused kernel
// (3 modes, 32-byte nonzeros with remap ids and write orders; R = 16, 32, 64;
// FP32 or BF16 factors).  U (nonzeros in flight per lane group) keeps each
// ring of row slices at 64 registers or fewer per lane.
#include "mttkrp_tile.cuh"

namespace spm {

template <typename T, int NV, int U>
static int tile_by_mode(const MttkrpArgs& a, cudaStream_t s) {
  switch (a.mode) {
    case 0: return launch_tile_kernel<T, NV, 0, U>(a, s);
    case 1: return launch_tile_kernel<T, NV, 1, U>(a, s);
    default: return launch_tile_kernel<T, NV, 2, U>(a, s);
  }
}

bool tile_form_supported(int nmodes, int es, int alpha_word, int R) {
  return nmodes == 3 && es == 32 && alpha_word > 0 && (R == 16 || R == 32 || R == 64);
}

int launch_mttkrp_tile(const MttkrpArgs& a, cudaStream_t s) {
  constexpr int U = kTileU, UH = kTileU / 2 > 0 ? kTileU / 2 : 1;
  if (a.dtype == SPM_DTYPE_BF16) {
    switch (a.R) {
      case 16: return tile_by_mode<__nv_bfloat16, 2, U>(a, s);
      case 32: return tile_by_mode<__nv_bfloat16, 4, U>(a, s);
      default: return tile_by_mode<__nv_bfloat16, 8, U>(a, s);
    }
  }
  switch (a.R) {
    case 16: return tile_by_mode<float, 2, U>(a, s);
    case 32: return tile_by_mode<float, 4, U>(a, s);
    default: return tile_by_mode<float, 8, UH>(a, s);
  }
}

}  // namespace spm
