// Host state of the gate network and the launchers shared by its
// translation units (inference in gate.cu, training in mlp_train.cu).
#pragma once
#include "ctx.cuh"
#include "gate.cuh"

// The opaque network handle of the C ABI.
struct spoly_mlp {
  int device = 0;
  spoly::DevBuf theta;   // FP32 master parameters [kParams]
  spoly::DevBuf adam_m;  // Adam first moments [kParams]
  spoly::DevBuf adam_v;  // Adam second moments [kParams]
  spoly::DevBuf packed;  // BF16 tensor-core operand tiles and FP32 vectors of inference [kPackWords]
  spoly::DevBuf status;  // inference status word (non-zero: a bounded wait gave up)
  long long wait_cycles = 0;  // limit of the inference's tensor-core waits (0: the default)
  int64_t adam_step = 0;
  // Training scratch (grown on demand).
  spoly::DevBuf xb, yb, z1, z2, z3, dz1, dz2, dz3, grad, loss, lists, list_n, logits;
};

namespace spoly {

// Gate inference over n rows: features from `feat` ([n][24] FP32) when it is
// non-null, else computed from `chains`.  Writes logits (if non-null) and
// appends the chains whose logit reaches tau_logit to out_chains (if
// non-null), counting them in *out_n.  *status (if non-null) becomes non-zero
// when a wait for the tensor core gave up; the outputs are then incomplete.
struct GateParams {
  MeshView mesh;
  QueryView qv;
  const int32_t* chains;
  const float* feat;
  int64_t n;
  const uint32_t* packed;
  float tau_logit;
  float* logits;
  int32_t* out_chains;
  unsigned long long* out_n;
  unsigned long long* status;
  long long wait_cycles;  // limit of each per-layer completion wait in SM cycles (<= 0: the default)
};

cudaError_t launch_gate(const GateParams& G, int num_sms, cudaStream_t st);
cudaError_t launch_pack(const float* theta, uint32_t* packed, cudaStream_t st);

}  // namespace spoly
