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
// h[s][j_x][j_y][m_z] (N^2 x N/2 complex per section, the collapse of the
// lifted correlation, as k_lift_collapse forms it from the two spectra) of the
// knots kA (unrotated) and kB (rotated by RB, row major, and mirrored in r),
// both spectra by the 4D NUFFT; cone = the cone transform table
// ((3 (N/2)^2 + 1) x N_r), slices = device sections, scale = P^-3 P_r^-1; ws of
// lift4_ws_bytes(N, Nr) bytes.  Synchronises s once per spectrum (to size its
// support box).
cudaError_t lift4_pair(const Lift4Tables &t, int N, int Nr, const float4 *kA, int nA, const float4 *kB, int nB,
                       const double (&RB)[9], double period, double period_r, const float2 *cone, const float *slices,
                       int nslices, float scale, void *ws, float2 *h, int nsm, cudaStream_t s);

} // namespace bc
