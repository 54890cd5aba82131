// field_internal.h -- grid helpers implemented in field.cu and tables.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/crp.h"

namespace crp {

size_t node_bytes(int dtype);
// Convert [N][3] values (src_dtype) on the device into node storage.
crp_status grid_pack(const void* src_dev, int src_dtype, int64_t N, int dtype, void* nodes,
                     cudaStream_t s);
// Convert node storage into [N][3] float64 on the device.
crp_status grid_unpack(const void* nodes, int dtype, int64_t N, double* dst_dev, cudaStream_t s);
// Per-cell records of a binary32 node grid: cell (i, j, k) holds the 8
// coefficients of its trilinear polynomial in the in-cell fractions (see
// field.cu), 24 floats in 8 float4 (the last two zero): one aligned
// 128-byte record per cell.
crp_status grid_cells(const void* nodes, const int64_t n[3], void* cells, cudaStream_t s);
// Generate the turbulent field of `d` into node storage (synchronises s).
crp_status grid_turbulence(const crp_grid_desc* d, void* nodes, cudaStream_t s);
// Gauss-Legendre nodes and weights on [-1, 1] (host).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
// Fill the three rate tables (device arrays of d->n doubles) by quadrature.
crp_status tables_compute(const crp_tables_desc* d, double* beta, double* pion, double* gdr,
                          cudaStream_t s);

}  // namespace crp
