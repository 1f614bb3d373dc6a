// Analytic initial data generated on the device, the pi-symmetry monitor
// (Sec. 3.2) and the symmetrisation of data.
#include "sacrak_dev.cuh"

namespace sacrak {

// SplitMix64 output function (Steele, Lea & Flood 2014) applied to state x
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform value in [-1, 1) of field f at level-global cell (i, j, k)
__device__ __forceinline__ double noise_value(uint64_t seed, int f, long long i, long long j,
                                              long long k) {
  uint64_t h = splitmix64(seed + (uint64_t)f);
  h = splitmix64(h ^ (uint64_t)i);
  h = splitmix64(h ^ (uint64_t)j);
  h = splitmix64(h ^ (uint64_t)k);
  return __dsub_rn(__dmul_rn(__dmul_rn((double)(h >> 11), 0x1.0p-53), 2.0), 1.0);
}

// Coordinates and arithmetic use explicitly rounded operations so that the
// values agree bit for bit with a plain left-to-right evaluation on the host.
__global__ void init_data_kernel(InitArgs A, int patch) {
  const DevPatch* P = A.patches + patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)P->NX * P->NY * P->NZ;
  if (id >= tot) return;
  const int I = id % P->NX, J = (id / P->NX) % P->NY, K = id / ((long long)P->NX * P->NY);
  const int idx[3] = {I, J, K};
  double x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    x[d] = __dadd_rn(P->origin[d], __dmul_rn((double)(idx[d] - GH) + 0.5, P->dx));
  double v[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) v[f] = flat_value(f);
  if (A.kind == 1) {
    double psi = 1.0;
    for (int a = 0; a < A.npunct; ++a) {
      double dx = __dsub_rn(x[0], A.pos[3 * a]);
      double dy = __dsub_rn(x[1], A.pos[3 * a + 1]);
      double dz = __dsub_rn(x[2], A.pos[3 * a + 2]);
      double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      double r = __dsqrt_rn(r2);
      psi = __dadd_rn(psi, __ddiv_rn(A.m[a], __dmul_rn(2.0, r)));
    }
    double W = __ddiv_rn(1.0, __dmul_rn(psi, psi));
    v[F_W] = W;
    v[F_ALP] = W;
  } else if (A.kind == 2) {
    const double pi = 3.141592653589793;
    double ph = 2.0 * pi * x[0] / A.gw_len;
    double H = 1.0 - A.gw_amp * sin(ph);
    double dH = -A.gw_amp * cos(ph) * 2.0 * pi / A.gw_len;
    double Kxx = -(pi * A.gw_amp / A.gw_len) * cos(ph) / sqrt(H);
    double K = Kxx / H;
    double W = pow(H, -1.0 / 6.0);
    v[F_W] = W;
    v[F_GXX] = pow(H, 2.0 / 3.0);
    v[F_GYY] = pow(H, -1.0 / 3.0);
    v[F_GZZ] = v[F_GYY];
    v[F_KH] = K;
    v[F_AXX] = 2.0 / 3.0 * W * W * Kxx;
    v[F_AYY] = -1.0 / 3.0 * W * W * K;
    v[F_AZZ] = v[F_AYY];
    v[F_GAMX] = 2.0 / 3.0 * pow(H, -5.0 / 3.0) * dH;
    v[F_ALP] = sqrt(H);
  }
  const long long q = I + (long long)J * P->px + (long long)K * P->plane;
  double* u = P->buf[A.levels[P->level].ring];
  if (A.noise_amp != 0.0) {
    long long gi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      gi[d] = (long long)llrint((P->origin[d] - A.lo[d]) / P->dx) + idx[d] - GH;
    for (int f = 0; f < NF; ++f)
      v[f] = __dadd_rn(v[f], __dmul_rn(A.noise_amp, noise_value(A.seed, f, gi[0], gi[1], gi[2])));
  }
  for (int f = 0; f < NF; ++f) u[f * P->fstride + q] = v[f];
}

// points with x < 0 (array index below NX/2 on a patch centred on x = y = 0)
// take the parity-signed value of their partner (-x, -y, z)
__global__ void symmetrise_kernel(const DevPatch* patches, const DevLevel* levels, int patch) {
  const DevPatch* P = patches + patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = P->NX / 2;
  const long long tot = (long long)half * P->NY * P->NZ;
  if (id >= tot) return;
  const int I = id % half, J = (id / half) % P->NY, K = id / ((long long)half * P->NY);
  double* u = P->buf[levels[P->level].ring];
  const long long q = I + (long long)J * P->px + (long long)K * P->plane;
  const long long qm = (P->NX - 1 - I) + (long long)(P->NY - 1 - J) * P->px + (long long)K * P->plane;
  for (int f = 0; f < NF; ++f) {
    double s = (double)pi_parity(f);
    u[f * P->fstride + q] = s * u[f * P->fstride + qm];
  }
}

// max |f - s_f f(mirror)| over all points and fields; block partial maxima
__global__ void pi_symmetry_kernel(const DevPatch* patches, const DevLevel* levels, int patch,
                                   double* partial) {
  __shared__ double red[8];
  const DevPatch* P = patches + patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)P->NX * P->NY * P->NZ;
  double mx = 0.0;
  if (id < tot) {
    const int I = id % P->NX, J = (id / P->NX) % P->NY, K = id / ((long long)P->NX * P->NY);
    const double* u = P->buf[levels[P->level].ring];
    const long long q = I + (long long)J * P->px + (long long)K * P->plane;
    const long long qm =
        (P->NX - 1 - I) + (long long)(P->NY - 1 - J) * P->px + (long long)K * P->plane;
    for (int f = 0; f < NF; ++f) {
      double d = fabs(u[f * P->fstride + q] - (double)pi_parity(f) * u[f * P->fstride + qm]);
      if (!(d <= mx)) mx = isnan(d) ? INFINITY : d;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    partial[blockIdx.x] = m;
  }
}

__global__ void max_partials_kernel(const double* partial, int n, double* out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) m = fmax(m, partial[b]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

void launch_init(const InitArgs& a, int patch, long long tot, cudaStream_t st) {
  init_data_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(a, patch);
}

void launch_symmetrise(const DevPatch* p, const DevLevel* l, int patch, long long half_tot,
                       cudaStream_t st) {
  symmetrise_kernel<<<(unsigned)((half_tot + 127) / 128), 128, 0, st>>>(p, l, patch);
}

int launch_pi_symmetry(const DevPatch* p, const DevLevel* l, int patch, long long tot,
                       double* partial, double* out, cudaStream_t st) {
  int nb = (int)((tot + 255) / 256);
  pi_symmetry_kernel<<<nb, 256, 0, st>>>(p, l, patch, partial);
  max_partials_kernel<<<1, 256, 0, st>>>(partial, nb, out);
  return nb;
}

}  // namespace sacrak
