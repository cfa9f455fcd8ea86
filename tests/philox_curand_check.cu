// Second independent Philox4x32-10 reference for the oracle's pin, on the
// GPU: reads lines "seed g attempt domain" and prints the four 32-bit
// outputs of cuRAND's device Philox block function for counter (g_lo, g_hi,
// domain, attempt) and key (seed_lo, seed_hi).
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void blocks(const unsigned long long* in, unsigned* out, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const unsigned long long seed = in[4 * t], g = in[4 * t + 1];
  const unsigned a = (unsigned)in[4 * t + 2], dom = (unsigned)in[4 * t + 3];
  const uint4 c = make_uint4((unsigned)g, (unsigned)(g >> 32), dom, a);
  const uint2 k = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
  const uint4 r = curand_Philox4x32_10(c, k);
  out[4 * t] = r.x;
  out[4 * t + 1] = r.y;
  out[4 * t + 2] = r.z;
  out[4 * t + 3] = r.w;
}

int main() {
  std::vector<unsigned long long> h;
  unsigned long long s, g, a, d;
  while (std::scanf("%llu %llu %llu %llu", &s, &g, &a, &d) == 4) {
    h.push_back(s);
    h.push_back(g);
    h.push_back(a);
    h.push_back(d);
  }
  const int n = (int)(h.size() / 4);
  if (n == 0) return 0;
  unsigned long long* din = nullptr;
  unsigned* dout = nullptr;
  if (cudaMalloc(&din, h.size() * 8) != cudaSuccess) return 2;
  if (cudaMalloc(&dout, (size_t)n * 16) != cudaSuccess) return 2;
  cudaMemcpy(din, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
  blocks<<<(n + 127) / 128, 128>>>(din, dout, n);
  std::vector<unsigned> r((size_t)n * 4);
  if (cudaMemcpy(r.data(), dout, r.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  for (int t = 0; t < n; ++t) std::printf("%u %u %u %u\n", r[4 * t], r[4 * t + 1], r[4 * t + 2], r[4 * t + 3]);
  cudaFree(din);
  cudaFree(dout);
  return 0;
}
