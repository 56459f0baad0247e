// The replica-batched FP32 colour pass specialised to one update policy (Sec. II; Sec. IV.C):
// when every site of a colour class has the same policy, the kernel is compiled for that
// policy alone, so a warp does not carry the other proposals' instructions. The attempt is
// the same code as the table-driven kernel's with the policy fixed at compile time, so the
// spins are bit for bit those of that kernel.
#include <cuda_runtime.h>

#include "vegas_r32.cuh"

namespace vegas {

PassFn select_r32_fixed(int pm, int lm, int code) {
#define VEGAS_R32_ROW(PM, LM)                                                                                    \
    {pass32_r32<PM, LM, 2 + kPolFlip>, pass32_r32<PM, LM, 2 + kPolSmallStep>, pass32_r32<PM, LM, 2 + kPolGaussian>, \
     pass32_r32<PM, LM, 2 + kPolHinzkeNowak>, pass32_r32<PM, LM, 2 + kPolAdaptive>, pass32_r32<PM, LM, 2 + kPolQIsing>}
    static const PassFn tab[3][3][6] = {
        {VEGAS_R32_ROW(0, 0), VEGAS_R32_ROW(0, 1), VEGAS_R32_ROW(0, 2)},
        {VEGAS_R32_ROW(1, 0), VEGAS_R32_ROW(1, 1), VEGAS_R32_ROW(1, 2)},
        {VEGAS_R32_ROW(2, 0), VEGAS_R32_ROW(2, 1), VEGAS_R32_ROW(2, 2)},
    };
#undef VEGAS_R32_ROW
    return tab[pm][lm][code - kPolFlip];
}

}  // namespace vegas
