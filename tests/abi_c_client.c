/* A plain C99 client of the C ABI (include/heat.h): it must compile as C with
 * warnings as errors, link against libheat.so and run without a GPU, since every
 * call below fails its argument checks before any device work. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "heat.h"

static int fails = 0;

static void expect(int got, int want, const char *what) {
  if (got != want) {
    printf("FAIL %s: %d (%s), want %d\n", what, got, heat_strerror(got), want);
    ++fails;
  }
}

int main(void) {
  heat_ctx *c = (heat_ctx *)&fails; /* must be reset to NULL on failure */
  expect(heat_create(&c, 0, 4, 0.5, 1.0, 1.0, HEAT_F64), HEAT_EINVAL, "nx = 0");
  if (c != NULL) {
    printf("FAIL context not reset on failure\n");
    ++fails;
  }
  expect(heat_create(&c, 10, 2, 0.5, 1.0, 0.0, HEAT_F64), HEAT_EINVAL, "dx = 0");
  expect(heat_create(&c, 10, 2, NAN, 1.0, 1.0, HEAT_F32C), HEAT_EINVAL, "k = NaN");
  expect(heat_create(NULL, 10, 2, 0.5, 1.0, 1.0, HEAT_F64), HEAT_EINVAL, "out = NULL");
  expect(heat_run(NULL, 1), HEAT_EINVAL, "heat_run(NULL)");
  expect(heat_set(NULL, NULL, 0), HEAT_EINVAL, "heat_set(NULL)");
  heat_batch *b = NULL;
  expect(heat_batch_create(&b, 0, HEAT_F64), HEAT_EINVAL, "batch capacity 0");
  heat_destroy(NULL);
  if (strlen(heat_strerror(HEAT_ETIMEOUT)) == 0) {
    printf("FAIL empty message\n");
    ++fails;
  }
  printf("%s\n", fails ? "failed" : "c client ok");
  return fails != 0;
}
