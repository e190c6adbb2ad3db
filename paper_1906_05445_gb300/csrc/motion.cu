// motion.cu -- the solids' motion for one step, on the device (Sec. 3.2).
//
// A lattice with a free solid keeps its solids' state in device memory, so
// that a step needs no read-back of the force record: one thread per solid
// reads the step's force and torque (and, under Kempe's treatment, the
// inside fluid's integrals of Eq. 24) and advances the velocities and the
// centre.  With dt = 1 and rho_f = rho0 = 1:
//  - bounce-back, Eq. 20: rho_p V dU = F + (rho_p - rho_f) V g, I dOmega = T,
//    F and T the momentum exchange of the step (Eq. 17);
//  - IBM, Eq. 23 (Feng & Michaelides): the force gains rho_f V (U^n - U^(n-1))
//    and the torque I (rho_f / rho_p)(Omega^n - Omega^(n-1));
//  - IBM, Eqs. 24-26 (Kempe et al.): instead the change over the step of the
//    inside fluid's integrals of u and r x u (the first step: no change);
//  - IBM, Eq. 22 (Uhlmann): dU = (F + (rho_p - rho_f) V g) / ((rho_p - rho_f) V),
//    dOmega = T / (I (1 - rho_f / rho_p)).
// The centre moves by the mean of the old and the new velocity.  V and I are
// those of a sphere (4/3 pi R^3, 2/5 m R^2) or a cylinder (pi R^2 times its
// length: 1 on a 2D lattice, nz on a 3D one; 1/2 m R^2 about z).  A solid
// with prescribed motion moves by its velocity.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr double kPi = 3.14159265358979323846;

// A moving solid keeps 1.5 spacings from a velocity or stress-free face and
// R + 5 from an outflow face (as lbm_set_domain requires); a violation is
// recorded for the next synchronising call.
__device__ void check_clearance(const MotionArgs &m, const SolidDev &b) {
  for (int a = 0; a < m.dim; a++) {
    if (m.face[2 * a] == LBM_FACE_PERIODIC) continue;
    if (a == 2 && b.kind == LBM_CYLINDER_Z) continue;
    const double mlo = m.face[2 * a] == LBM_FACE_CONVECTIVE ? b.R + 5.0 : b.R + 1.5;
    const double mhi = m.face[2 * a + 1] == LBM_FACE_CONVECTIVE ? b.R + 5.0 : b.R + 1.5;
    if (b.c[a] - mlo < 0 || b.c[a] + mhi > m.len[a] - 1) *m.err = 1;
  }
}

__global__ void k_motion(const MotionArgs m) {
  const int k = threadIdx.x;
  if (k >= m.n) return;
  SolidDev &b = m.now->s[k];
  FreeDev &f = m.fr[k];
  const double R = b.R;
  if (!(f.rho_p > 0)) {
    for (int a = 0; a < 3; a++) b.c[a] += b.U[a];
    if (b.U[0] != 0 || b.U[1] != 0 || b.U[2] != 0) check_clearance(m, b);
    return;
  }
  const bool cyl = m.dim == 2 || b.kind == LBM_CYLINDER_Z;
  const double V = cyl ? kPi * R * R * (m.dim == 2 ? 1.0 : (double)m.nz)
                       : 4.0 / 3.0 * kPi * R * R * R;
  const double mass = f.rho_p * V, I = mass * (cyl ? 0.5 : 0.4) * R * R;
  const double *rec = m.rec + 6 * k;
  const double *In = m.kempe ? m.kempe + 6 * k : nullptr;
  double Un[3], On[3];
  for (int a = 0; a < 3; a++) {
    double dv = rec[a] + (f.rho_p - 1.0) * V * f.g[a];
    double dw = rec[3 + a];
    if (m.mode == MM_IBM_KEMPE) {
      if (!f.have_Ip) {
        f.Ip[a] = In[a];
        f.Ip[3 + a] = In[3 + a];
      }
      dv += In[a] - f.Ip[a];
      dw += In[3 + a] - f.Ip[3 + a];
    } else if (m.mode == MM_IBM_FENG) {
      dv += V * (b.U[a] - f.Up[a]);
      dw += I / f.rho_p * (b.Om[a] - f.Omp[a]);
    }
    if (m.mode == MM_IBM_UHLMANN) {
      Un[a] = b.U[a] + dv / ((f.rho_p - 1.0) * V);
      On[a] = b.Om[a] + dw / (I * (1.0 - 1.0 / f.rho_p));
      continue;
    }
    Un[a] = b.U[a] + dv / mass;
    On[a] = b.Om[a] + dw / I;
  }
  if (m.dim == 2) Un[2] = 0;
  if (cyl) On[0] = On[1] = 0;
  if (m.mode == MM_IBM_KEMPE) {
    for (int c = 0; c < 6; c++) f.Ip[c] = In[c];
    f.have_Ip = 1;
  }
  for (int a = 0; a < 3; a++) {
    b.c[a] += 0.5 * (b.U[a] + Un[a]);
    f.Up[a] = b.U[a];
    f.Omp[a] = b.Om[a];
    b.U[a] = Un[a];
    b.Om[a] = On[a];
  }
  check_clearance(m, b);
}

}  // namespace

void launch_motion(const MotionArgs &m, cudaStream_t st) {
  if (m.n > 0) k_motion<<<1, 32, 0, st>>>(m);
}

}  // namespace lbm
