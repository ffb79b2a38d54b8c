// Instantiations of the launch helpers for FP64 storage.
#include "ops_impl.cuh"
using namespace tsm;
TSM_INSTANTIATE_STORAGE(F64)
TSM_INSTANTIATE_PAIR(F64, F64)
TSM_INSTANTIATE_CONVERT(F64, F32)
TSM_INSTANTIATE_CONVERT(F64, F64)
