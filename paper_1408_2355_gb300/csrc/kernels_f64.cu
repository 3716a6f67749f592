// float64 specialisations of the hot-path kernels (lanes per row 1..16,
// padded-ELL widths 8 and 16).
#include "kernels.cuh"

namespace segimpl {

bool get_kernels_f64(int lpr, int w, KernelSet* ks) {
  switch (lpr) {
    case 1: return fill_kernels_w<double, 1>(w, ks);
    case 2: return fill_kernels_w<double, 2>(w, ks);
    case 4: return fill_kernels_w<double, 4>(w, ks);
    case 8: return fill_kernels_w<double, 8>(w, ks);
    case 16: return fill_kernels_w<double, 16>(w, ks);
    default: return false;
  }
}

}  // namespace segimpl
