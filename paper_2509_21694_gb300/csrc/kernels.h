// Launch interfaces of the evaluator's kernels.
#pragma once

#include "common.cuh"
#include "edge_math.cuh"

namespace mp {

// One message-passing layer over a receiver-sorted CSR (local ids).
struct EdgeArgs {
    int64_t n;
    const int64_t* row_ptr;
    const int32_t* col;
    const int8_t* shift;
    const double* x;          // [n][3] wrapped positions
    // tensor-core kernels: per edge of this CSR, (u_x, u_y, u_z, r) of
    // d = x_j - x_i + n L (launch_edge_geometry)
    const float4* geo;
    EdgeConst k;
    const LayerW* w;
    const float* Hin;         // [n][NLM][F] layer input features
    float* Aout;              // forward: [n][NLM][F] aggregated messages (/N_avg)
    const float* Alpha;       // adjoint: [n][NLM][F] dE/dA / N_avg
    const float* Gout;        // adjoint: [n][NLM][F] dE/d(layer output)
    float* Gin;               // adjoint: [n][NLM][F] dE/d(layer input); null at layer 0
    const uint8_t* seed;      // adjoint: root flags (null = all 1)
    double* frc;              // adjoint: [n][3] forces, accumulated
    bool first;               // layer 0: input l >= 1 features are zero
    int* err;                 // device error word (bit 2: bounded wait timed out)
    int* sched;               // tensor-core kernels: row-group counter (zeroed per launch)
    // adjoint, optional: per-row virial sum_e g_e (x) d_e of the pair gradients
    // g_e added to the row's force, component-major [9][vir_stride], accumulated
    double* vir;
    int64_t vir_stride;
    // adjoint: rows < n_recv receive messages at this layer; an edge whose two
    // ends are both >= n_recv has zero adjoint on both sides and may be
    // skipped (<= 0: every row is a receiver)
    int64_t n_recv;
    // BF16 layer 0 by hidden unit (tensor-core path): local species of every
    // row, the embedding table [S][F], and scratch [n][S][NLM][H] for the
    // forward's per-row sums G and the adjoint's per-atom vectors V (null:
    // the channel-wise kernels are used)
    const int32_t* species;
    const float* emb;
    int n_species;
    float* vfirst;
};

// (u_x, u_y, u_z, r) of every edge of a CSR over n rows, for the tensor-core
// edge kernels, formed once per evaluation: the positions x [n][3] are split
// into FP32 pairs (scratch `split`, 2 n float4) and each edge vector is
// formed from them in FP32 arithmetic.
int launch_edge_geometry(int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const int8_t* shift, const double* x, const EdgeConst& k, float4* geo,
                         float4* split, cudaStream_t st);
int launch_edge_fwd_f32(const Model& m, const EdgeArgs& a, cudaStream_t st);
int launch_edge_bwd_f32(const Model& m, const EdgeArgs& a, cudaStream_t st);
int launch_edge_fwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms);
int launch_edge_bwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms);

// Node update of layer t: S = W0 A0 + sum_l Ul Bl + b; h0' = h0 + silu(S);
// hl' = hl + Vl Al (skipped when last).
struct NodeArgs {
    int64_t n;
    const LayerW* w;
    const float* A;
    const float* Hin;
    float* Hout;
    float* S;
    const float* Gout;   // adjoint
    float* Alpha;        // adjoint output (/N_avg)
    float inv_navg;
    bool first;          // layer 0: input features with l >= 1 are zero (not stored)
    bool last;
    int* err;            // device error bits (tensor-core kernels)
};
int launch_node_fwd_f32(const Model& m, const NodeArgs& a, cudaStream_t st);
int launch_node_bwd_f32(const Model& m, const NodeArgs& a, cudaStream_t st);
// BF16 operands on tcgen05 (F = 128, lmax = 2).  The adjoint splits its
// per-partition operand into three BF16 parts, so it stays linear to FP32
// rounding.
int launch_node_fwd_bf16(const Model& m, const NodeArgs& a, cudaStream_t st, int num_sms);
int launch_node_bwd_bf16(const Model& m, const NodeArgs& a, cudaStream_t st, int num_sms);

// Tangent (forward-mode) pass of one layer along a displacement field v.
struct TangentArgs {
    int64_t n;
    const int64_t* row_ptr;
    const int32_t* col;
    const int8_t* shift;
    const double* x;          // [n][3] wrapped positions
    const float* v;           // [n][3] displacement field
    EdgeConst k;
    const LayerW* w;
    const float* Hin;         // [n][NLM][F] layer input values
    const float* dHin;        // [n][NLM][F] layer input tangents (ignored at layer 0)
    float* dAout;             // edge kernel output: message tangents (/N_avg)
    const float* A;           // node kernel: layer messages
    const float* dA;          // node kernel: message tangents
    const float* S;           // node kernel: pre-activations
    float* dHout;             // node kernel output: layer output tangents
    bool first, last;
};
int launch_edge_tangent_f32(const Model& m, const TangentArgs& a, cudaStream_t st);
int launch_node_tangent_f32(const Model& m, const TangentArgs& a, cudaStream_t st);

}  // namespace mp
