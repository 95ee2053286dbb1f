// Test driver for tests/test_gpu_half_product.py: the FP16 form's roundings from the
// decoder's device header.  Mode "product": out[i] = half_product(a[i], b[i]) (the
// check-to-variable rounding of alpha m); mode "quotient": out[i] =
// half_of_quotient(a[i], b[i]) (the merge's rounding of num / P).
// Input file: int32 N, float32 a[N], float32 b[N]; output file: float32 out[N].
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#include "nms_device.cuh"

__global__ void half_round_kernel(const float *a, const float *b, float *out, int N, int quotient) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N)
    out[i] = quotient ? __half2float(bchlib::half_of_quotient(a[i], b[i])) : bchlib::half_product(a[i], b[i]);
}

int main(int argc, char **argv) {
  if (argc != 4) return 2;
  const int quotient = argv[3][0] == 'q' ? 1 : 0;
  FILE *fi = std::fopen(argv[1], "rb");
  if (!fi) return 2;
  int N = 0;
  if (std::fread(&N, 4, 1, fi) != 1 || N <= 0) return 2;
  std::vector<float> a(N), m(N), o(N);
  if (std::fread(a.data(), 4, N, fi) != size_t(N) || std::fread(m.data(), 4, N, fi) != size_t(N)) return 2;
  std::fclose(fi);
  float *da = nullptr, *dm = nullptr, *dout = nullptr;
  if (cudaMalloc(&da, 4 * size_t(N)) != cudaSuccess || cudaMalloc(&dm, 4 * size_t(N)) != cudaSuccess ||
      cudaMalloc(&dout, 4 * size_t(N)) != cudaSuccess)
    return 3;
  cudaMemcpy(da, a.data(), 4 * size_t(N), cudaMemcpyHostToDevice);
  cudaMemcpy(dm, m.data(), 4 * size_t(N), cudaMemcpyHostToDevice);
  half_round_kernel<<<(N + 255) / 256, 256>>>(da, dm, dout, N, quotient);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return 4;
  cudaMemcpy(o.data(), dout, 4 * size_t(N), cudaMemcpyDeviceToHost);
  FILE *fo = std::fopen(argv[2], "wb");
  if (!fo) return 2;
  std::fwrite(o.data(), 4, N, fo);
  std::fclose(fo);
  cudaFree(da);
  cudaFree(dm);
  cudaFree(dout);
  return 0;
}
