/* A plain C program against include/hopf.h and libhopf_gb300.so: option
 * defaults, argument validation and an empty batch, none of which touches a
 * device.  Prints "ok" and exits 0 when every check holds. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "hopf.h"

#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            printf("failed: %s (line %d): %s\n", #cond, __LINE__,     \
                   hopf_last_error());                                \
            return 1;                                                 \
        }                                                             \
    } while (0)

int main(void) {
    /* double integrator: A = [[0, 1], [0, 0]], B = [0; 1], box |u| <= 1,
       target radius 0.1 (W = 0.01 I) */
    const double A[4] = {0.0, 1.0, 0.0, 0.0}, B[2] = {0.0, 1.0}, hw[1] = {1.0};
    const double W[4] = {0.01, 0.0, 0.0, 0.01}, Wbad[4] = {1.0, 2.0, 2.0, 1.0};
    hopf_problem prob;
    memset(&prob, 0, sizeof prob);
    prob.n = 2;
    prob.m = 1;
    prob.A = A;
    prob.B = B;
    prob.ctrl_kind = HOPF_BOX;
    prob.half_widths = hw;
    prob.W = W;

    hopf_opts o;
    hopf_default_opts(&o);
    CHECK(o.N == 100 && o.gap_every == 8 && o.tol_gap == 1e-5 && o.rule == HOPF_LEFT_RIEMANN);
    o.host_io = 1;

    float x[4] = {1.0f, 0.5f, -1.0f, 0.3f}, t[1] = {1.0f};
    float phi[2], ps[4], gap[2];
    int iters[2], status[2], steps = -1;

    /* an empty batch needs no device */
    CHECK(hopf_value(&prob, &o, 0, x, t, 0, NULL, phi, ps, gap, iters, status, NULL) == HOPF_SUCCESS);
    CHECK(hopf_time_to_reach(&prob, &o, 0, x, NULL, NULL, NULL, t, ps, gap, status, &steps, NULL) ==
          HOPF_SUCCESS && steps == 0);

    /* validation happens before any device work */
    prob.W = Wbad;
    CHECK(hopf_value(&prob, &o, 2, x, t, 0, NULL, phi, ps, gap, iters, status, NULL) == HOPF_ENOTSPD);
    prob.W = W;
    o.tau = -1.0;
    CHECK(hopf_value(&prob, &o, 2, x, t, 0, NULL, phi, ps, gap, iters, status, NULL) == HOPF_EINVAL);
    o.tau = 1.0;
    o.rule = HOPF_LEFT_FIXED;                    /* needs terminal-time variables */
    CHECK(hopf_value(&prob, &o, 2, x, t, 0, NULL, phi, ps, gap, iters, status, NULL) == HOPF_EINVAL);
    o.variables = HOPF_VARS_TERMINAL;
    o.t_max = INFINITY;                          /* and a finite t_max */
    CHECK(hopf_value(&prob, &o, 2, x, t, 0, NULL, phi, ps, gap, iters, status, NULL) == HOPF_EINVAL);
    o.t_max = 2.0;
    CHECK(hopf_value(&prob, &o, 0, x, t, 0, NULL, phi, ps, gap, iters, status, NULL) == HOPF_SUCCESS);
    o.rule = HOPF_LEFT_RIEMANN;
    o.tol_T = 1e-17;                             /* below float64 resolution */
    CHECK(hopf_time_to_reach(&prob, &o, 2, x, NULL, NULL, NULL, t, ps, gap, status, &steps, NULL) == HOPF_EINVAL);

    CHECK(strcmp(hopf_status_string(HOPF_OK), "ok") == 0);
    printf("ok\n");
    return 0;
}
