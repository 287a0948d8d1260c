// hj_r1_inst.cuh -- launchers of the one-thread-per-pair kernels (hj_r1.cuh)
// for one padded dimension C, and their registration in the launcher table.
#pragma once

#include "hj_internal.h"
#include "hj_r1.cuh"

namespace hjd {

template <int C>
cudaError_t launch_r1_eval(const void *a, int grid, cudaStream_t s)
{
    r1::k_eval<C><<<grid, BLOCK, 0, s>>>(*(const RowArgs<float> *)a);
    return cudaGetLastError();
}
template <int C>
cudaError_t launch_r1_grad(const void *a, int grid, cudaStream_t s)
{
    r1::k_grad<C><<<grid, BLOCK, 0, s>>>(*(const RowArgs<float> *)a);
    return cudaGetLastError();
}
template <int C>
cudaError_t launch_r1_phi64(const void *a, int grid, cudaStream_t s)
{
    r1::k_phi64<C><<<grid, BLOCK, 0, s>>>(*(const CertArgs<float> *)a);
    return cudaGetLastError();
}
template <int C, int MODE, int TPP>
cudaError_t launch_r1_desc(const void *a, int grid, cudaStream_t s)
{
    r1::k_desc<C, MODE, TPP><<<grid, BLOCK, 0, s>>>(*(const DescArgs<float> *)a);
    return cudaGetLastError();
}

template <int C>
void register_r1(Registry &r)
{
    KSet &k = r.r1[C];
    k.eval = &launch_r1_eval<C>;
    k.f_eval = (const void *)&r1::k_eval<C>;
    k.grad = &launch_r1_grad<C>;
    k.f_grad = (const void *)&r1::k_grad<C>;
    k.cd = &launch_r1_desc<C, DESC_CD, 1>;
    k.f_cd = (const void *)&r1::k_desc<C, DESC_CD, 1>;
    k.gd = &launch_r1_desc<C, DESC_GD, 1>;
    k.f_gd = (const void *)&r1::k_desc<C, DESC_GD, 1>;
    k.gd_lat = &launch_r1_desc<C, DESC_GD, 2>;
    k.cert_final = &launch_r1_phi64<C>;
    k.f_cert_final = (const void *)&r1::k_phi64<C>;
    k.f_gd_lat = (const void *)&r1::k_desc<C, DESC_GD, 2>;
}

}  // namespace hjd
