// sg_qnet.cu -- dueling Q-network, fused eps-greedy rollout, replay ring.
#include "sg_host.h"

int sg_rollout_eps_q(sg_sim* sim, int K, sg_qnet* q, const float* eps, sg_replay* rp, float* obs, float* obs_seq,
                     uint8_t* act_seq, float* rew_seq, uint8_t* done_seq, cudaStream_t stream) {
  (void)sim; (void)K; (void)q; (void)eps; (void)rp; (void)obs; (void)obs_seq; (void)act_seq; (void)rew_seq; (void)done_seq;
  (void)stream;
  return SG_E_INVAL;
}
