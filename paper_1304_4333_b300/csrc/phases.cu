// Simulator phases (temporary: entry points not yet implemented return SPS_ERR_UNSUPPORTED).
#include "common.cuh"

extern "C" {
sps_status sps_loglik_grad(sps_ctx*, const double*, int64_t, int64_t, double*, double*, int32_t) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_state_create(sps_ctx*, int32_t, int32_t, uint64_t, sps_state** out) { if (out) *out = nullptr; return SPS_ERR_UNSUPPORTED; }
void sps_state_destroy(sps_state* st) { delete st; }
sps_status sps_state_get(sps_ctx*, const sps_state*, double*, double*, double*, int64_t*, double*) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_state_set(sps_ctx*, sps_state*, const double*, const double*, int64_t) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_cphase(sps_ctx*, sps_state*, int64_t, int64_t*, double*, double*) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_sphase(sps_ctx*, sps_state*, const double*, int32_t*, int32_t) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_mstep(sps_ctx*, sps_state*, int32_t, const double*, double*, sps_mstep_info*) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_mphase(sps_ctx*, sps_state*, int32_t, int32_t, int32_t*, double*, double*) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_run(sps_ctx*, int32_t, int32_t, const sps_schedule*, sps_schedule*, sps_result*) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_resample(sps_ctx*, const double*, const double*, int32_t, int32_t, int32_t*, int32_t) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_philox(sps_ctx*, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, int64_t, uint32_t*, int32_t) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_ess(sps_ctx*, const double*, int64_t, int32_t, double*, double*, int32_t) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_particle_cov(sps_ctx*, const double*, int64_t, double*, int32_t) { return SPS_ERR_UNSUPPORTED; }
sps_status sps_rw_step_given(sps_ctx*, double*, double*, int64_t, int64_t, const double*, const double*, const double*, int32_t, double*, int32_t*, int32_t) { return SPS_ERR_UNSUPPORTED; }
}
