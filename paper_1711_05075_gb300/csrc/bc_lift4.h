// Lifted spectrum by a 4D type-1 NUFFT (bc_lift_nufft.cu), for the lifted
// correlation (bc_lift.cu).  Not part of the public interface.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace bc {

// Tables built by
// launch_build_tables for the spatial axes (N modes, n = 2N) and the lifted
// axis (N_r modes, n_r = 2 N_r), window width 8.
struct Lift4Tables {
    float *deconv_s = nullptr, *deconv_r = nullptr; // 1 / phi^ in FFT order: N, N_r entries
    float2 *tw_s = nullptr, *tw_r = nullptr;        // exp(-2 pi i k / n), k < n; the same for n_r
    float *consts = nullptr;                        // window polynomials (Tables::consts layout)
    int *dbox = nullptr;                            // support box of a shape: 8 device words
    int *hbox = nullptr;                            // and their page-locked host copy
};
size_t lift4_ws_bytes(int N, int Nr);
// rho (N^2 x N/2 x N_r, overwritten) = the spectrum of Eq. (rhoAhat) of the n
// knots (x, y, z, r) rotated by R (row major) and, with mirror, r -> -r; ws of
// lift4_ws_bytes(N, Nr) bytes.  Synchronises s once (to size the support box).
cudaError_t lift4_spectrum(const Lift4Tables &t, int N, int Nr, const float4 *knots, int n, const double (&R)[9],
                           int mirror, double period, double period_r, void *ws, float2 *rho, int nsm, cudaStream_t s);

} // namespace bc
