// Fused aggregation kernels for the guidance bases B_GRAY8, B_GRAY9.
#include "hgf_fused.cuh"

HGF_INSTANTIATE_BASIS(hgf::B_GRAY8)
HGF_INSTANTIATE_BASIS(hgf::B_GRAY9)
