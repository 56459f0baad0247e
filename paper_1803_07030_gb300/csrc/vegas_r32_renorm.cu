// The replica-batched FP32 colour pass of a step's last class-1 pass with the end-of-step
// renormalisation |S_i| = s_i folded in (two colour classes, every class-1 link to class 0):
// the spins it leaves equal those of the same pass followed by the renormalisation pass.
#include <cuda_runtime.h>

#include "vegas_r32.cuh"

namespace vegas {

PassFn select_r32_renorm(int pm) {
    static const PassFn tab[3] = {pass32_r32<0, 1, 0, 1>, pass32_r32<1, 1, 0, 1>, pass32_r32<2, 1, 0, 1>};
    return tab[pm < 0 ? 0 : (pm > 2 ? 2 : pm)];
}

}  // namespace vegas
