// Instantiations of the launch helpers for FP32 storage.
#include "ops_impl.cuh"
using namespace tsm;
TSM_INSTANTIATE_STORAGE(F32)
TSM_INSTANTIATE_PAIR(F32, F32)
TSM_INSTANTIATE_CONVERT(F32, F64)
TSM_INSTANTIATE_CONVERT(F32, F32)
