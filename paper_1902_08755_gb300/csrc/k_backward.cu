// k_backward.cu -- gradients of the compositing operators (placeholder until
// the kernels land; every entry point reports EC_ERR_UNSUPPORTED).
#include "ec_internal.cuh"

extern "C" {

ec_status ec_composite_alpha_backward(ec_ctx*, const ec_image*, const int32_t*, int32_t, ec_rect,
                                      const float*, void* const*, int32_t, ec_stream_t)
{
    return EC_ERR_UNSUPPORTED;
}

ec_status ec_composite_alpha_fwd_bwd(ec_ctx*, const ec_image*, const int32_t*, int32_t,
                                     const ec_target*, float*, const float*, void* const*, int32_t,
                                     ec_rect*, ec_stream_t)
{
    return EC_ERR_UNSUPPORTED;
}

ec_status ec_composite_depth_backward(ec_ctx*, const int16_t*, ec_rect, const float*, int32_t,
                                      const ec_rect*, const int32_t*, float* const*, ec_stream_t)
{
    return EC_ERR_UNSUPPORTED;
}

}
