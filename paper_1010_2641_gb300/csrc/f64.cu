// Plain FP64 GPU kernel of Eq. 2: one thread per S point, a straight loop
// over the atoms in double precision with sincospi, no centring and no
// splitting of S.  It is the GPU comparator the FP32 paths are measured
// against (the paper notes FP64 runs on fewer units, Section 2.3).
#include <cuda_runtime.h>
#include "device_common.cuh"
#include "launch.h"

namespace scatter {

struct F64Args {
  const double* xyz;
  const float* occ;
  const int32_t* slot_src;
  const Segment* segs;
  const int32_t* inst_seg_off;  // [batch+1] segment range of each instance
  const int32_t* s_inst;        // LIST batch: instance of each point, or null
  const double* coef64;
  const double* ftab64;         // Eq. 4 factor table [n_species][M][2], or null
  int64_t n_s;
  const double* S64;            // LIST [M][3]
  const double* axis64;         // GRID [n0 | n1 | n2]
  int64_t n0, n1, n2;
  int grid;
  double inv4a2;
  float2* out_amp;
  float* out_int;
};

__device__ __forceinline__ void form_factor64(const double* cf, double s2, double* re, double* im) {
  double f0 = cf[8];
  for (int i = 0; i < 4; ++i) f0 += cf[i] * exp(-cf[4 + i] * s2);
  const double dw = exp(-cf[11] * s2);
  *re = (f0 + cf[9]) * dw;
  *im = cf[10] * dw;
}

__global__ void __launch_bounds__(128) k_f64(const F64Args a) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.n_s) return;
  double S[3];
  if (a.grid) {
    const int64_t i2 = m % a.n2, line = m / a.n2, i1 = line % a.n1, i0 = line / a.n1;
    S[0] = a.axis64[i0];
    S[1] = a.axis64[a.n0 + i1];
    S[2] = a.axis64[a.n0 + a.n1 + i2];
  } else {
    S[0] = a.S64[3 * m];
    S[1] = a.S64[3 * m + 1];
    S[2] = a.S64[3 * m + 2];
  }
  const int b = a.s_inst ? a.s_inst[m] : 0;
  const double s2 = (S[0] * S[0] + S[1] * S[1] + S[2] * S[2]) * a.inv4a2;
  double are = 0.0, aim = 0.0;
  for (int g = a.inst_seg_off[b]; g < a.inst_seg_off[b + 1]; ++g) {
    const Segment sg = a.segs[g];
    double fr, fi;
    if (a.ftab64) {
      fr = a.ftab64[2 * ((int64_t)sg.species * a.n_s + m)];
      fi = a.ftab64[2 * ((int64_t)sg.species * a.n_s + m) + 1];
    } else {
      form_factor64(a.coef64 + kNCoef * sg.species, s2, &fr, &fi);
    }
    double tr = 0.0, ti = 0.0;
    for (int64_t slot = sg.begin; slot < sg.end; ++slot) {
      const int32_t j = a.slot_src[slot];
      if (j < 0) continue;
      const double* r = a.xyz + 3 * (int64_t)j;
      const double w = a.occ ? (double)a.occ[j] : 1.0;
      const double ph = S[0] * r[0] + S[1] * r[1] + S[2] * r[2];
      double sn, cs;
      sincospi(2.0 * ph, &sn, &cs);
      tr += w * cs;
      ti += w * sn;
    }
    are += fr * tr - fi * ti;
    aim += fr * ti + fi * tr;
  }
  if (a.out_amp) a.out_amp[m] = make_float2((float)are, (float)aim);
  if (a.out_int) a.out_int[m] = (float)(are * are + aim * aim);
}

scatter_status launch_f64(scatter_plan_t p, const double* xyz, const float* occ, float2* amp_out,
                          float* int_out, cudaStream_t st) {
  if (p->n_s == 0) return SCATTER_OK;
  F64Args a{};
  a.xyz = xyz;
  a.occ = occ;
  a.slot_src = p->d.slot_src;
  a.segs = p->d.segs;
  a.inst_seg_off = p->d.chunk_seg_off;  // one chunk per instance on this path
  a.s_inst = p->d.s_inst;
  a.coef64 = p->d.coef64;
  a.ftab64 = p->d.ftab64;
  a.n_s = p->n_s;
  a.S64 = p->d.S64;
  a.axis64 = p->d.axis64;
  a.n0 = p->n_axis[0];
  a.n1 = p->n_axis[1];
  a.n2 = p->n_axis[2];
  a.grid = p->s_kind == SCATTER_S_GRID;
  a.inv4a2 = 1.0 / (4.0 * p->lattice_a * p->lattice_a);
  a.out_amp = amp_out;
  a.out_int = int_out;
  const int64_t nb = (p->n_s + 127) / 128;
  timing_begin(p, st);
  k_f64<<<(unsigned)nb, 128, 0, st>>>(a);
  timing_end(p, st);
  p->last_launches += 1;
  return cuda_status(cudaGetLastError(), "fp64 kernel launch");
}

}  // namespace scatter
