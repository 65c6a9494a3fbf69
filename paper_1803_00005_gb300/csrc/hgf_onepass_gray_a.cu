// Single-pass aggregation kernels for gray powers I..I^d, d = 1..5.
#include "hgf_onepass.cuh"

HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY1)
HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY2)
HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY3)
HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY4)
HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY5)
