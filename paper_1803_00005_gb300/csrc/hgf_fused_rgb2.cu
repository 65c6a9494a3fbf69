// Fused aggregation kernels for the guidance bases B_RGB_MONO2.
#include "hgf_fused.cuh"

HGF_INSTANTIATE_BASIS(hgf::B_RGB_MONO2)
