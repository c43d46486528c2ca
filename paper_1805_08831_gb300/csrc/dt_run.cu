// dt_run: command-line driver of the C ABI for profiling (no Python).
//   dt_run N [steps] [seed]            one cloud of N points
//   dt_run batch C [steps] [seed]      C clouds, sizes round(exp(U[ln 50, ln 50000]))
//   dt_run deg N [steps] [seed]        the degenerate mix of N points
// Points are i.i.d. uniform in the unit cube (a SplitMix64 stream, as in the package's synthetic
// generator), or the degenerate mix of that generator's recipe: 40 % on the sphere inscribed in
// the unit cube (normalised Box-Muller directions), 40 % in 64 Gaussian clusters (sigma 0.01),
// 20 % on the lattice {0..99}^3 / 99. Runs `steps` triangulations on one handle and prints the
// tetrahedron count, the device time of each step and the handle's counters.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <string>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../include/dt.h"

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Value i (0-based) of the SplitMix64 stream of `seed`, and the uniform double in [0, 1) from it.
static uint64_t stream(uint64_t seed, uint64_t i) { return mix64((seed << 32) + (i + 1) * 0x9E3779B97F4A7C15ull); }
static double uni(uint64_t seed, uint64_t i) { return (double)(stream(seed, i) >> 11) * (1.0 / 9007199254740992.0); }
static double gauss(uint64_t seed, uint64_t i) {  // Box-Muller, cosine branch, on uniforms 2i and 2i + 1
  const double u1 = 1.0 - uni(seed, 2 * i), u2 = uni(seed, 2 * i + 1);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.141592653589793 * u2);
}

static void degenerate_mix(uint64_t n, uint64_t seed, std::vector<double>& xyz) {
  const uint64_t n_sph = (2 * n) / 5, n_clu = (2 * n) / 5, n_lat = n - n_sph - n_clu;
  for (uint64_t i = 0; i < n_sph; ++i) {
    double g[3], r = 0;
    for (int k = 0; k < 3; ++k) {
      g[k] = gauss(seed, 3 * i + k);
      r += g[k] * g[k];
    }
    r = std::sqrt(r);
    if (r == 0.0) r = 1.0;
    for (int k = 0; k < 3; ++k) xyz[3 * i + k] = 0.5 + 0.5 * (g[k] / r);
  }
  for (uint64_t i = 0; i < n_clu; ++i)
    for (int k = 0; k < 3; ++k)
      xyz[3 * (n_sph + i) + k] = uni(seed + 1, 3 * (i % 64) + k) + 0.01 * gauss(seed + 2, 3 * i + k);
  for (uint64_t i = 0; i < n_lat; ++i)
    for (int k = 0; k < 3; ++k) xyz[3 * (n_sph + n_clu + i) + k] = (double)(stream(seed + 3, 3 * i + k) % 100) / 99.0;
}

int main(int argc, char** argv) {
  const bool batch = argc > 1 && std::string(argv[1]) == "batch";
  const bool deg = argc > 1 && std::string(argv[1]) == "deg";
  const int a0 = (batch || deg) ? 2 : 1;
  uint64_t n = argc > a0 ? (uint64_t)std::atof(argv[a0]) : 1000000;
  int steps = argc > a0 + 1 ? std::atoi(argv[a0 + 1]) : 1;
  uint64_t seed = argc > a0 + 2 ? std::strtoull(argv[a0 + 2], nullptr, 10) : 2;
  std::vector<uint64_t> off;
  if (batch) {
    const uint32_t clouds = (uint32_t)n;
    off.assign(clouds + 1, 0);
    for (uint32_t c = 0; c < clouds; ++c) {
      double u = (double)(mix64((seed << 40) + (c + 1) * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
      off[c + 1] = off[c] + (uint64_t)std::llround(std::exp(std::log(50.0) + u * (std::log(50000.0) - std::log(50.0))));
    }
    n = off[clouds];
  }
  std::vector<double> xyz(3 * n);
  if (deg) {
    degenerate_mix(n, seed, xyz);
  } else {
    for (uint64_t i = 0; i < 3 * n; ++i) xyz[i] = uni(seed, i);
  }
  double* d = nullptr;
  if (cudaMalloc(&d, 24 * n) != cudaSuccess) return 2;
  cudaMemcpy(d, xyz.data(), 24 * n, cudaMemcpyHostToDevice);
  dt_config cfg{};
  cfg.seed = seed;
  dt_handle* h = nullptr;
  int rc = dt_create(&h, &cfg);
  if (rc) return 3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int s = 0; s < steps; ++s) {
    dt_clear(h);
    cudaEventRecord(e0);
    rc = batch ? dt_batch(h, d, off.data(), (uint32_t)(off.size() - 1)) : dt_insert(h, d, n);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    uint64_t T = 0;
    dt_get_tets(h, nullptr, 0, &T, nullptr, 0);
    std::printf("step %d rc %d ms %.2f tets %llu Mtets/s %.2f\n", s, rc, ms, (unsigned long long)T, T / ms / 1e3);
    if (rc) break;
  }
  dt_stats st{};
  dt_get_stats(h, &st);
  std::printf("rounds %llu passes %llu attempts %llu conflicts %llu launches %llu\n",
              (unsigned long long)st.n_rounds, (unsigned long long)st.n_passes,
              (unsigned long long)st.n_attempts, (unsigned long long)st.n_conflicts,
              (unsigned long long)st.n_launches);
  std::printf("async launches %llu restarts %llu handoffs %llu walk steps %llu big %llu exact %llu ms_sort %.2f "
              "ms_first %.2f device bytes %llu\n",
              (unsigned long long)st.n_async, (unsigned long long)st.n_restarts,
              (unsigned long long)st.n_exact_handoff, (unsigned long long)st.sum_walk,
              (unsigned long long)st.n_big, (unsigned long long)st.n_exact, st.ms_sort, st.ms_first_round,
              (unsigned long long)st.device_bytes);
  dt_destroy(h);
  cudaFree(d);
  return rc ? 1 : 0;
}
