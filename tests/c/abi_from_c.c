/* A plain C11 caller of libjmg.so: it includes only the public headers and
 * exercises the host-side part of the ABI (defaults, workspace sizes, status
 * strings, illegal-argument codes), which needs no GPU.  Prints "ok" and
 * exits 0 when every check holds, else names the first failed check. */
#include <stdio.h>
#include <string.h>

#include "jmg.h"
#include "jmg_dev.h"

#define CHECK(cond)                                   \
  do {                                                \
    if (!(cond)) {                                    \
      printf("failed: %s (line %d)\n", #cond, __LINE__); \
      return 1;                                       \
    }                                                 \
  } while (0)

int main(void) {
  jmg_options o;
  jmg_default_options(&o);
  CHECK(o.nb == 128 && o.prec == JMG_PREC_NATIVE && o.maxit == 300 && o.tol == 1e-13);

  /* plain solves need only their tickets; the mixed ones hold the FP32 factor */
  CHECK(jmg_workspace_size(JMG_OP_POTRF, 1000, 1, JMG_F64, &o) == 0);
  size_t plain = jmg_workspace_size(JMG_OP_POSV, 1000, 4, JMG_F64, &o);
  CHECK(plain > 0 && plain % 256 == 0);
  jmg_options m = o;
  m.prec = JMG_PREC_FP16;
  m.words = 2;
  CHECK(jmg_workspace_size(JMG_OP_POSV, 1000, 4, JMG_F64, &m) >= (size_t)4 * 1000 * 1000);
  /* the host-buffer call stages A (n x n) and B (n x nrhs) in front */
  CHECK(jmg_workspace_size(JMG_OP_POSV_HOST, 1000, 4, JMG_F64, &o) ==
        (size_t)8 * 1000 * 1000 + 32000 + 256 + plain);

  CHECK(strcmp(jmg_status_string(JMG_ERR_NOT_SPD), "matrix is not positive definite") == 0);
  CHECK(strcmp(jmg_status_string(-3), "illegal argument") == 0);

  /* LAPACK-style argument codes, returned before anything touches a device */
  int dummy = 0;
  CHECK(jmg_potrf(-1, NULL, 1, JMG_F64, &dummy, NULL, NULL, 0, NULL) == -1);
  CHECK(jmg_potrs(4, 1, NULL, 3, NULL, 4, JMG_F64, NULL, 0, NULL) == -4);
  CHECK(jmg_posv(4, 1, NULL, 4, NULL, 4, JMG_F64, NULL, NULL, NULL, NULL, 0, NULL) == -8);
  CHECK(jmg_posv_batched(129, 1, 1, &dummy, 129, 129 * 129, &dummy, 129, 129, JMG_F64, &dummy,
                         NULL) == JMG_ERR_UNSUPPORTED);
  double a[4] = {4, 2, 2, 3}, b[2] = {1, 1}, x[2] = {0, 0};
  int info = -5;
  CHECK(jmg_posv_host(2, 1, a, 1, b, 2, x, 2, JMG_F64, &info, NULL, NULL, NULL, 0, NULL) == -4);
  CHECK(jmg_posv_host(2, 1, a, 2, b, 2, x, 2, JMG_F64, &info, NULL, NULL, NULL, 0, NULL) ==
        JMG_ERR_WORKSPACE);
  CHECK(info == 0);
  CHECK(jmg_dev_residual_workspace(1000, 4) >= jmg_dev_residual_workspace(100, 4));
  printf("ok\n");
  return 0;
}
