/* A plain C11 program against include/btrace.h and libbtrace.so: the
 * boundary is a C ABI (no C++ in the header, stable struct layouts) usable
 * without Python.  It makes no compute call, so it runs without a GPU:
 * defaults, argument checks and a context request that fails cleanly when no
 * device is present.  Exit status 0 when every check holds; the failing check
 * is printed otherwise. */
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "btrace.h"

static int failures = 0;
#define CHECK(cond)                                              \
  do {                                                           \
    if (!(cond)) {                                               \
      fprintf(stderr, "c_abi_check: failed: %s (line %d)\n", #cond, __LINE__); \
      failures++;                                                \
    }                                                            \
  } while (0)

int main(int argc, char **argv) {
  int expect_no_device = argc > 1 && strcmp(argv[1], "--no-device") == 0;
  /* layouts: every field of the parameters is 4 bytes wide, the stats are
   * 14 int64 counters then 3 doubles */
  CHECK(sizeof(bt_trace_params) == 4 * (1 + BT_MAX_BANDS + 1 + 1 + 2 + 1 + 1 + 1 + 1 + 1 + 1));
  CHECK(offsetof(bt_trace_params, air_atten_db_per_m) == 4);
  CHECK(offsetof(bt_trace_params, queue_depth) == sizeof(bt_trace_params) - 4);
  CHECK(sizeof(bt_stats) == 8 * 17);
  CHECK(offsetof(bt_stats, trace_ms) == 8 * 14);

  bt_trace_params p;
  memset(&p, 0xff, sizeof(p));
  CHECK(bt_params_default(&p) == BT_OK);
  CHECK(p.max_order == 4 && p.tiles_x == 1 && p.tiles_y == 1 && p.precision == BT_PREC_MIXED);
  CHECK(p.t_eps_m == 1e-3f && p.watchdog_ms == 2000 && p.chunk_beams == 0 && p.queue_depth == 0);
  for (int b = 0; b < BT_MAX_BANDS; b++) CHECK(p.air_atten_db_per_m[b] == 0.0f);
  CHECK(bt_params_default(NULL) == BT_E_INVALID);

  /* every entry point refuses a NULL context without touching a device */
  CHECK(bt_destroy(NULL) == BT_OK);
  CHECK(bt_create(NULL, 0, NULL) == BT_E_INVALID);
  CHECK(bt_load_scene(NULL, NULL, 0, NULL, 0, NULL, NULL, 0, 0, NULL) == BT_E_INVALID);
  CHECK(bt_unload_scene(NULL, 0) == BT_E_INVALID);
  CHECK(bt_set_sources(NULL, 0, NULL, NULL, 0, 0) == BT_E_INVALID);
  CHECK(bt_set_directivity(NULL, 0, NULL, 0, NULL) == BT_E_INVALID);
  CHECK(bt_beam_axes(NULL, 0, NULL) == BT_E_INVALID);
  CHECK(bt_set_microphones(NULL, 0, NULL, 0) == BT_E_INVALID);
  CHECK(bt_trace(NULL, 0, &p) == BT_E_INVALID);
  CHECK(bt_submit(NULL, 0, &p) == BT_E_INVALID);
  CHECK(bt_poll(NULL, 0) == BT_E_INVALID);
  CHECK(bt_wait(NULL, 0) == BT_E_INVALID);
  CHECK(bt_read_levels(NULL, 0, NULL, NULL, NULL, NULL) == BT_E_INVALID);
  CHECK(bt_cast_rays(NULL, 0, NULL, NULL, NULL, 0, 1e-3f, NULL, NULL) == BT_E_INVALID);
  CHECK(bt_trace_noalloc(NULL, 0, &p, NULL, NULL) == BT_E_INVALID);
  CHECK(bt_batch_create(NULL, NULL, 0, NULL, NULL) == BT_E_INVALID);
  CHECK(bt_set_result(NULL, 0, NULL, NULL) == BT_E_INVALID);
  CHECK(bt_scene_share(NULL, 0, NULL) == BT_E_INVALID);
  CHECK(bt_trace_ranges(NULL, 0, NULL, NULL, NULL, NULL, 0) == BT_E_INVALID);
  CHECK(bt_ranges_stats(NULL, NULL) == BT_E_INVALID);
  CHECK(bt_batch_run(NULL) == BT_E_INVALID);
  CHECK(bt_batch_stats(NULL, NULL) == BT_E_INVALID);
  CHECK(bt_batch_destroy(NULL) == BT_OK);
  CHECK(strcmp(bt_last_error(NULL), "null context") == 0);
  CHECK(bt_kernel_launches() == 0);

  if (expect_no_device) {
    bt_ctx *ctx = (bt_ctx *)&p; /* must be overwritten */
    CHECK(bt_create(&ctx, 0, NULL) == BT_E_CUDA);
    CHECK(ctx == NULL);
    CHECK(bt_kernel_launches() == 0);
  }
  if (failures == 0) printf("c_abi_check: ok\n");
  return failures == 0 ? 0 : 1;
}
