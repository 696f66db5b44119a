// Host FP64 tables (Daubechies filters, DCT-II matrix) of the MUFFIN library.
#pragma once

namespace muffin {

// h[0 .. 2p-1]: extremal-phase Daubechies scaling filter db<p>, sum sqrt(2).
void daubechies_lowpass(int p, double *h);

// C[k*L + l] = c_k cos(pi (2l+1) k / (2L)), orthonormal DCT-II.
void dct2_matrix(int L, double *C);

// ||W||^2 of the J-scale starlet (B3 spline, periodic) on the n x n grid:
// max over the DFT frequencies of sum_j (A_j - A_{j+1})^2 + A_J^2, A_j the
// transfer function of the first j smoothings.
double iuwt_norm2(int n, int J);

}  // namespace muffin
