// Instantiations of the launch helpers for BF16 storage (a unit of its own so
// that the two 16-bit tiers compile in parallel).
#include "ops_impl.cuh"
using namespace tsm;
TSM_INSTANTIATE_STORAGE(BF16)
TSM_INSTANTIATE_PAIR(BF16, F32)
TSM_INSTANTIATE_CONVERT(F32, BF16)
TSM_INSTANTIATE_CONVERT(BF16, F32)
TSM_INSTANTIATE_CONVERT(F64, BF16)
TSM_INSTANTIATE_CONVERT(BF16, F64)
TSM_INSTANTIATE_CONVERT(BF16, BF16)
