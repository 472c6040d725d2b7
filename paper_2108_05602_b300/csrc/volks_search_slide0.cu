// Instantiations of the FP32 search kernel's sliding-segment form for the
// power-of-two bands, rate padding 0.
#include "search_kernel.cuh"

namespace vk {
VK_POW2_VARIANTS(VK_SEARCH_INST_SLIDE, 0)
}  // namespace vk
