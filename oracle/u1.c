/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Compact U(1) gauge links with the axion coupling (section "ALP-gauge
 * interactions", Eq. AxionInfEOM).  Placeholder until that sector is written.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

double orc_u1_magnetic_sum(int N, const double* links) { (void)N; (void)links; return 0.0; }

void orc_u1_rk_step(const orc_model* m, int scheme, double h,
                    double* phi, double* pi, double* links, double* efield, double* abt)
{
    (void)m; (void)scheme; (void)h; (void)phi; (void)pi; (void)links; (void)efield; (void)abt;
}

void orc_u1_gauss(const orc_model* m, const double* phi, const double* links,
                  const double* efield, double a, double* out_gauss)
{
    (void)m; (void)phi; (void)links; (void)efield; (void)a; (void)out_gauss;
}
