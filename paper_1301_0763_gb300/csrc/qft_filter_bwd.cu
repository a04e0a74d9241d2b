// qft_filter_bwd.cu -- the backward kernels of the spectral-filter layer
// (the sources are those of qft_filter.cu; compiled separately, in parallel).
#define QFT_FILTER_BACKWARD_TU 1
#include "qft_filter.cu"
