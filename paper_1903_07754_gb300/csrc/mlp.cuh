// Cost model of the learned switch (not in the paper: it replaces the fixed
// fullness threshold and the fixed Wedge Frontier precision of Section 3.4 by
// a prediction of each candidate's iteration time).
//
// Network: 12 features -> 64 (ReLU) -> 64 (ReLU) -> 1, predicting the
// natural log of the milliseconds that the next iteration (transformation +
// pull) takes under a candidate.  Candidates: dense pull, or pull over the
// Wedge Frontier at coarsening k = 0..4.
//
// Flat parameter layout (FP32 master, 5057 floats):
//   W1[64][12] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3
#pragma once

#include <math.h>
#include <stdint.h>

namespace wedge {

constexpr int kMlpIn = 12;
constexpr int kMlpHidden = 64;
constexpr int kMlpW1 = 0;
constexpr int kMlpB1 = kMlpW1 + kMlpHidden * kMlpIn;        // 768
constexpr int kMlpW2 = kMlpB1 + kMlpHidden;                  // 832
constexpr int kMlpB2 = kMlpW2 + kMlpHidden * kMlpHidden;     // 4928
constexpr int kMlpW3 = kMlpB2 + kMlpHidden;                  // 4992
constexpr int kMlpB3 = kMlpW3 + kMlpHidden;                  // 5056
constexpr int kMlpParams = kMlpB3 + 1;                       // 5057
constexpr int kCandidates = 6;                               // dense, sparse k = 0..4

// Graph statistics that enter every feature vector, and the band of
// fullness / E inside which the decision evaluates the model (outside it the
// traces' unanimous choice: the Wedge Frontier at k = 0 below, dense above).
struct GraphFeat {
    float log2V, log2E, avg_deg, skew, app;
    float band_lo, band_hi;
};

// Features of one candidate for the iteration that pulls frontier F_t:
//  1 log2(|F_t|+1)/32        2 log2(fullness+1)/32    3 fullness/E
//  4 log2(rowsum+1)/32       5 log2(V)/32             6 log2(E)/32
//  7 (E/V)/64                8 log2(1 + max/mean outdeg)/16
//  9 t/(t+8)                 10 app (BFS 0, CC 0.5, SSSP 1)
//  11 candidate is sparse    12 candidate k / 4
__host__ __device__ inline void mlp_features(const GraphFeat& gf, double E, unsigned nfront, double fullness,
                                             unsigned rowsum, unsigned it, int cand, float* x) {
    x[0] = (float)(log2((double)nfront + 1.0) / 32.0);
    x[1] = (float)(log2(fullness + 1.0) / 32.0);
    x[2] = (float)(E > 0 ? fullness / E : 0.0);
    x[3] = (float)(log2((double)rowsum + 1.0) / 32.0);
    x[4] = gf.log2V / 32.0f;
    x[5] = gf.log2E / 32.0f;
    x[6] = gf.avg_deg / 64.0f;
    x[7] = gf.skew;
    x[8] = (float)((double)it / ((double)it + 8.0));
    x[9] = gf.app;
    x[10] = cand > 0 ? 1.0f : 0.0f;
    x[11] = cand > 0 ? (float)(cand - 1) / 4.0f : 0.0f;
}

}  // namespace wedge
