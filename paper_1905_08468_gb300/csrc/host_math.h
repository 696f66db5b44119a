// Host FP64 tables (Daubechies filters, DCT-II matrix) of the MUFFIN library.
#pragma once

namespace muffin {

// h[0 .. 2p-1]: extremal-phase Daubechies scaling filter db<p>, sum sqrt(2).
void daubechies_lowpass(int p, double *h);

// C[k*L + l] = c_k cos(pi (2l+1) k / (2L)), orthonormal DCT-II.
void dct2_matrix(int L, double *C);

}  // namespace muffin
