// nlms.h - argument blocks and launchers of the adaptive canceller's kernels.
//
// The feedback canceller (Sec. 5, Eq. 3) can adapt its sub-filter spectra
// F_hat once per block with a partitioned-block frequency-domain NLMS step
// (an extension: the paper's F_hat is static).  With P microphones, L
// loudspeakers, K_fb partitions, block B and the error e of the current
// microphone block:
//   E_p      = R2C_2B([0_B | e_p])
//   pow[k]   = lam pow[k] + (1 - lam) sum_l |U_l,0[k]|^2
//   F_hat[p][l][j][k] += mu E_p[k] conj(U_l,j[k]) / (K_fb pow[k] + delta)
// where U_l,j is delay-line entry j of loudspeaker l before this block's
// loudspeaker spectrum is pushed.  Packed bin 0 carries DC and Nyquist as two
// real bins, each with its own power.  FP32 storage only.
#pragma once
#include <cuda_runtime.h>

namespace gbconv {

// Error spectra, power recursion and the step-scaled error G = mu E / (K pow + delta).
struct NlmsPrepArgs {
    const float* e;        // [P][B] error block
    const float2* U;       // canceller delay-line ring, FP32 [n_kt][K][L][BT]
    int slot0;             // ring slot of delay-line entry 0 (newest loudspeaker spectrum)
    const float2* pow_in;  // [B] packed power (bin 0: (DC, Nyquist); else (pow, 0))
    float2* pow_out;       // [B] recursion result (written by CTA 0; a different buffer than pow_in)
    float2* G;             // [P][B] packed step-scaled error spectra
    int B, log2B, BT, L, K;
    float mu, lam, delta;
    const float2* tw;      // W_2B^j, j in [0, 2B)
};

// F_hat += G conj(U) over every (bin tile, output tile) filter tile.
struct NlmsUpdateArgs {
    float2* F;          // canceller filter spectra, tiles at (kt*n_lt + lt)*tile_elems, then [r][LTt][BT]
    const float2* U;    // delay-line ring [n_kt][K][L][BT]
    const float2* G;    // [P][B]
    int B, BT, n_kt, LT, n_lt, P, L, K, slot0;
    int rows_per_cta;   // reduction indices r = j*L + l per CTA
    size_t tile_elems;
};

cudaError_t launch_nlms_prep(const NlmsPrepArgs& a, int P, cudaStream_t s);
cudaError_t launch_nlms_update(const NlmsUpdateArgs& a, cudaStream_t s);

}  // namespace gbconv
