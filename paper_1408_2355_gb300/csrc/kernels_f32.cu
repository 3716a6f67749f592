// float32-storage specialisations of the hot-path kernels (lanes per row 1..8).
#include "kernels.cuh"

namespace segimpl {

bool get_kernels_f32(int lpr, KernelSet* ks) {
  switch (lpr) {
    case 1: return fill_kernels<float, 1>(ks);
    case 2: return fill_kernels<float, 2>(ks);
    case 4: return fill_kernels<float, 4>(ks);
    case 8: return fill_kernels<float, 8>(ks);
    default: return false;
  }
}

}  // namespace segimpl
