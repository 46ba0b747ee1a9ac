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
//
// Deferred update.  Write U_m for the loudspeaker spectra of block m, G_m for
// block m's step-scaled error (the factor of conj(U) above) and F_m for the
// spectra after block m's step, so F_m[j] = F_{m-1}[j] + G_m conj(U_{m-1-j}).
// The step is linear, so the prediction of block n,
//   c_n = sum_l F_n[0] U_n + sum_l sum_{j>=1} F_n[j] U_{n-j},
// equals the head with the current F_n[0], plus the tail with the spectra
// two steps old, plus two correlation terms:
//   sum_l sum_{j>=1} F_{n-2}[j] U_{n-j} + G_n A1_n + G_{n-1} A2_n,
//   A1_n = sum_l sum_{j>=1} conj(U_{l,n-1-j}) U_{l,n-j}   (lag one)
//   A2_n = sum_l sum_{j>=1} conj(U_{l,n-2-j}) U_{l,n-j}   (lag two).
// So nlms_prep applies the step to partition 0 at once, while the tail
// partitions take block m's step only during block m+1, in the same pass as
// the tail MAC of block m+2 (nlms_update_mac); that pass and the
// correlations (nlms_corr) need only delay-line entries up to block n-1, so
// both run on background streams a whole block ahead, as the static
// canceller's tail does.
// The two entries the pushes have overwritten by then are kept in a
// two-slot side buffer (by block parity) that the pack kernel fills.
#pragma once
#include <cuda_runtime.h>

namespace gbconv {

// Error spectra, power recursion, the step-scaled error G = mu E / (K pow +
// delta), and the step on partition 0 of the stored spectra.
struct NlmsPrepArgs {
    const float* e;        // [P][B] error block
    const float2* U;       // canceller delay-line ring, FP32 [n_kt][K][L][BT]
    int slot0;             // ring slot of delay-line entry 0 (newest loudspeaker spectrum)
    const float2* pow_in;  // [B] packed power (bin 0: (DC, Nyquist); else (pow, 0))
    float2* pow_out;       // [B] recursion result (written by CTA 0; a different buffer than pow_in)
    float2* G;             // [P][B] packed step-scaled error spectra
    int B, log2B, BT, L, K;
    float mu, lam, delta;
    const float2* tw;      // W_2B^j, j in [0, 2B), rounded to FP32
    const float2* tw_lo;   // W_2B^j - tw[j], rounded to FP32 (the float-float residual)
    // filter spectra, tiles at (kt*n_lt + lt)*tile_elems, then [r][LTt][BT]:
    // rows r = l (partition 0) take the step here
    float2* F;
    int LT, n_lt;
    size_t tile_elems;
};

// F_hat += G conj(U) over the reduction indices r = j*L + l in [r_begin, L*K)
// of every (bin tile, output tile) filter tile.
struct NlmsUpdateArgs {
    float2* F;          // canceller filter spectra, tiles at (kt*n_lt + lt)*tile_elems, then [r][LTt][BT]
    const float2* U;    // delay-line ring [n_kt][K][L][BT]
    const float2* G;    // [P][B]
    int B, BT, n_kt, LT, n_lt, P, L, K, slot0;
    int r_begin;        // L: partition 0 took the step in nlms_prep
    int rows_per_cta;   // reduction indices per CTA
    size_t tile_elems;
    // [n_kt][L][BT] spectra of entries j = K-1 (U_old[0]) and j = K-2
    // (U_old[1]) whose ring slots already hold newer blocks, or null (ring)
    const float2* U_old[2];
};

// Block m's step on the tail partitions (as NlmsUpdateArgs, r_begin = L)
// fused with the tail MAC of block m+2, which needs F_m: every stored
// spectrum is read once, takes the step (none when u.G is null), is written
// back and multiplied by its delay-line entry for the MAC.
struct NlmsUpdateMacArgs {
    NlmsUpdateArgs u;
    float2* partial;  // [S][P][B] split partials (the canceller's output kernel sums them)
    int S;            // splits of the rows [r_begin, L*K), one CTA row each
    int mac_slot0;    // ring slot of the MAC's entry 0 (block m+2); entry j at (mac_slot0 + j) mod K
};

// Chunks of the two correlations of block m+1, after block m's push:
//   A1[c][k] = sum_l sum_{j in chunk c} conj(U_{l,m-j}[k]) U_{l,m+1-j}[k]
//   A2[c][k] = sum_l sum_{j in chunk c} conj(U_{l,m-1-j}[k]) U_{l,m+1-j}[k]
// over j = 1..K-1 split into C chunks.  U_{m-i} sits at ring slot
// (slot_m + i) mod K for i < K; U_{m-K} (the last A2 term) in `oldest`.
// Packed bin 0: (DC, Nyquist) products.  K >= 2.
// The CTA that completes a bin range last (a ticket counter per range, reset
// by that CTA) sums the range's C chunks in order into A1f / A2f.
struct NlmsCorrArgs {
    const float2* U;       // ring [n_kt][K][L][BT]
    const float2* oldest;  // [n_kt][L][BT] block m-K
    float2* A1;            // [C][B]
    float2* A2;            // [C][B]
    float2* A1f;           // [B] sum of the chunks
    float2* A2f;           // [B]
    unsigned* ticket;      // [B] zero-initialised counters (one per bin range used)
    int B, BT, L, K, slot_m, C;
};

// Chunks of the correlations (at most 8).
int nlms_corr_chunks(int K);

cudaError_t launch_nlms_prep(const NlmsPrepArgs& a, int P, cudaStream_t s);
cudaError_t launch_nlms_update(const NlmsUpdateArgs& a, cudaStream_t s);
cudaError_t launch_nlms_corr(const NlmsCorrArgs& a, cudaStream_t s);
cudaError_t launch_nlms_update_mac(const NlmsUpdateMacArgs& a, cudaStream_t s);

}  // namespace gbconv
