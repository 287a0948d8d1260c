// hj_inst.cuh -- explicit instantiation of the kernels of one
// (precision, family, principle) for a list of components-per-thread C,
// and their registration in the launcher table.
#pragma once

#include "hj_internal.h"
#include "hj_kernels.cuh"

namespace hjd {

template <typename T, int C, int FAM, int PR>
cudaError_t launch_eval(const void *a, int grid, cudaStream_t s)
{
    k_eval<T, C, FAM, PR><<<grid, BLOCK, 0, s>>>(*(const RowArgs<T> *)a);
    return cudaGetLastError();
}
template <typename T, int C, int FAM, int PR>
cudaError_t launch_grad(const void *a, int grid, cudaStream_t s)
{
    k_grad<T, C, FAM, PR><<<grid, BLOCK, 0, s>>>(*(const RowArgs<T> *)a);
    return cudaGetLastError();
}
template <typename T, int C, int FAM, int PR, int MODE>
cudaError_t launch_desc(const void *a, int grid, cudaStream_t s)
{
    k_desc<T, C, FAM, PR, MODE><<<grid, BLOCK, 0, s>>>(*(const DescArgs<T> *)a);
    return cudaGetLastError();
}
template <typename Tv, int C, int FAM, int PR, int MODE>
cudaError_t launch_cert(const void *a, int grid, cudaStream_t s)
{
    k_cert<Tv, C, FAM, PR, MODE><<<grid, BLOCK, 0, s>>>(*(const CertArgs<Tv> *)a);
    return cudaGetLastError();
}

template <typename T>
constexpr int prec_index() { return sizeof(T) == 8 ? 1 : 0; }

// Descent, evaluation and gradient kernels for each C in the pack.
template <typename T, int FAM, int PR, int... Cs>
void register_compute(Registry &r)
{
    ((r.k[prec_index<T>()][FAM][PR][Cs].eval = &launch_eval<T, Cs, FAM, PR>,
      r.k[prec_index<T>()][FAM][PR][Cs].f_eval = (const void *)&k_eval<T, Cs, FAM, PR>,
      r.k[prec_index<T>()][FAM][PR][Cs].grad = &launch_grad<T, Cs, FAM, PR>,
      r.k[prec_index<T>()][FAM][PR][Cs].f_grad = (const void *)&k_grad<T, Cs, FAM, PR>,
      r.k[prec_index<T>()][FAM][PR][Cs].cd = &launch_desc<T, Cs, FAM, PR, DESC_CD>,
      r.k[prec_index<T>()][FAM][PR][Cs].f_cd = (const void *)&k_desc<T, Cs, FAM, PR, DESC_CD>,
      r.k[prec_index<T>()][FAM][PR][Cs].gd = &launch_desc<T, Cs, FAM, PR, DESC_GD>,
      r.k[prec_index<T>()][FAM][PR][Cs].f_gd = (const void *)&k_desc<T, Cs, FAM, PR, DESC_GD>,
      r.k[prec_index<T>()][FAM][PR][Cs].cg = &launch_desc<T, Cs, FAM, PR, DESC_CG>,
      r.k[prec_index<T>()][FAM][PR][Cs].f_cg = (const void *)&k_desc<T, Cs, FAM, PR, DESC_CG>),
     ...);
}

// FP64 certificate kernels reading v of type Tv, for each C in the pack.
template <typename Tv, int FAM, int PR, int... Cs>
void register_cert(Registry &r)
{
    ((r.k[prec_index<Tv>()][FAM][PR][Cs].cert_rows = &launch_cert<Tv, Cs, FAM, PR, 0>,
      r.k[prec_index<Tv>()][FAM][PR][Cs].f_cert_rows = (const void *)&k_cert<Tv, Cs, FAM, PR, 0>,
      r.k[prec_index<Tv>()][FAM][PR][Cs].cert_pairs = &launch_cert<Tv, Cs, FAM, PR, 1>,
      r.k[prec_index<Tv>()][FAM][PR][Cs].f_cert_pairs = (const void *)&k_cert<Tv, Cs, FAM, PR, 1>,
      r.k[prec_index<Tv>()][FAM][PR][Cs].cert_final = &launch_cert<Tv, Cs, FAM, PR, 2>,
      r.k[prec_index<Tv>()][FAM][PR][Cs].f_cert_final = (const void *)&k_cert<Tv, Cs, FAM, PR, 2>),
     ...);
}

}  // namespace hjd
