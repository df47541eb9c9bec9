/* The boundary as a C caller sees it: include/bmg.h compiled as strict C99,
 * linked against libbmg.so, and the calls that need no GPU exercised (error
 * strings, argument checks that fail before any device call, the build
 * variant query).  Prints one line per check; exits 0 when all hold. */
#include <stdio.h>
#include <string.h>

#include "bmg.h"

static int fails = 0;

static void check(int ok, const char* what) {
  printf("%s %s\n", ok ? "ok" : "FAIL", what);
  if (!ok) ++fails;
}

int main(void) {
  bmg_hierarchy* h = NULL;
  bmg_stencil st;
  bmg_opts o;
  memset(&o, 0, sizeof o);
  st.kind = 9;
  st.coef = NULL;
  check(strcmp(bmg_strerror(BMG_OK), "ok") == 0, "bmg_strerror(BMG_OK)");
  check(strcmp(bmg_strerror(BMG_EBOUNDS), "debug bounds check failed") == 0, "bmg_strerror(BMG_EBOUNDS)");
  check(bmg_setup(&st, 127, 127, &o, &h) == BMG_EINVAL && h == NULL, "bmg_setup rejects a NULL stencil");
  check(bmg_setup(&st, 0, 127, NULL, &h) == BMG_EINVAL, "bmg_setup rejects a bad size");
  check(strlen(bmg_last_error()) > 0, "bmg_last_error names the failure");
  check(bmg_solve(NULL, NULL, NULL, 1e-10, 10, NULL, NULL) == BMG_EINVAL, "bmg_solve rejects NULL");
  check(bmg_debug_build() == 0, "release library");
  bmg_free(NULL);
  return fails ? 1 : 0;
}
