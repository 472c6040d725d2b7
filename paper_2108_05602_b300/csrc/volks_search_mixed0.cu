// Instantiations of the FP32 search kernel for the bands of 3 * 2^a
// frequency points (mixed-radix delay FFTs), rate padding 0.
#include "search_kernel.cuh"

namespace vk {
VK_MIXED_VARIANTS(VK_SEARCH_INST, 0)
}  // namespace vk
