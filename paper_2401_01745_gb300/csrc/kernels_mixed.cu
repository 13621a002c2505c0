// Mixed-precision instantiations: z, the ionic model, the gating exponentials
// and the SpMV in FP32; V as a float-float pair; the power iteration forms
// q J v in FP32 (dual numbers for f_S) and accumulates norms in FP64.
#include "kernels.cuh"

namespace emrkc {

bool get_kernels_mixed(int model, KernelSet* ks) {
  switch (model) {
    case 0: Kernels<ModelNone<double>, ModelNone<float>, float, float, true, ModelNone<Dual>>::fill(ks, model); return true;
    case 1:
      Kernels<ModelPassive<double>, ModelPassive<float>, float, float, true, ModelPassive<Dual>>::fill(ks, model);
      return true;
    case 2: Kernels<ModelHH<double>, ModelHH<float>, float, float, true, ModelHH<Dual>>::fill(ks, model); return true;
    case 3:
      Kernels<ModelTTP06<double>, ModelTTP06<float>, float, float, true, ModelTTP06<Dual>>::fill(ks, model);
      return true;
    default: return false;
  }
}

}  // namespace emrkc
