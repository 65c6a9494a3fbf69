// Fused aggregation kernels for the guidance bases B_GRAY6, B_GRAY7.
#include "hgf_fused.cuh"

HGF_INSTANTIATE_BASIS(hgf::B_GRAY6)
HGF_INSTANTIATE_BASIS(hgf::B_GRAY7)
