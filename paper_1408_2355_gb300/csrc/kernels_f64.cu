// float64 specialisations of the hot-path kernels (lanes per row 1..16).
#include "kernels.cuh"

namespace segimpl {

bool get_kernels_f64(int lpr, KernelSet* ks) {
  switch (lpr) {
    case 1: return fill_kernels<double, 1>(ks);
    case 2: return fill_kernels<double, 2>(ks);
    case 4: return fill_kernels<double, 4>(ks);
    case 8: return fill_kernels<double, 8>(ks);
    case 16: return fill_kernels<double, 16>(ks);
    default: return false;
  }
}

}  // namespace segimpl
