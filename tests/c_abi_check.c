/* A plain C11 program against include/btrace.h and libbtrace.so: the
 * boundary is a C ABI (no C++ in the header, stable struct layouts) usable
 * without Python.  By default it makes no compute call, so it runs without a
 * GPU: defaults, argument checks and (with --no-device) a context request that
 * fails cleanly when no device is present.  With --trace it also traces one
 * source over a ground plane on device 0 and checks every microphone against
 * the closed form of Section 2's image-source method: the direct path plus the
 * ground image, r W / (4 pi d'^2).  Exit status 0 when every check holds; the
 * failing check is printed otherwise. */
#include <math.h>
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

/* One source 1.7 m above a 2 km ground square (energy coefficient 0.7),
 * level-4 beams, reflection order 2, microphones 5-30 m away at 3-20 m
 * height: every microphone lies in one direct and one ground-reflected beam
 * (the image direction is at least 8 degrees below the horizon, clear of the
 * beams that straddle it). */
static void trace_ground_plane(void) {
  bt_ctx *ctx = NULL;
  int rc = bt_create(&ctx, 0, NULL);
  CHECK(rc == BT_OK);
  if (rc != BT_OK) return;
  const float verts[4][3] = {{-1000, -1000, 0}, {1000, -1000, 0}, {1000, 1000, 0}, {-1000, 1000, 0}};
  const int32_t tris[2][3] = {{0, 1, 2}, {0, 2, 3}};
  const uint8_t mat[2] = {0, 0};
  float refl[BT_MAX_BANDS];
  float power[BT_MAX_BANDS];
  for (int b = 0; b < BT_MAX_BANDS; b++) {
    refl[b] = 0.7f;
    power[b] = 0.25f * (float)(b + 1);
  }
  const float src[3] = {1.3f, -2.1f, 1.7f};
  enum { NM = 6 };
  const float mics[NM][3] = {{12.5f, 3.25f, 3.5f}, {-7.75f, 20.5f, 11.0f}, {4.5f, -26.0f, 19.5f},
                             {-18.25f, -9.5f, 6.75f}, {25.0f, 14.5f, 15.25f}, {-3.5f, 8.75f, 4.25f}};
  int32_t sid = -1;
  CHECK(bt_load_scene(ctx, &verts[0][0], 4, &tris[0][0], 2, mat, refl, 1, BT_MAX_BANDS, &sid) == BT_OK);
  CHECK(bt_set_sources(ctx, sid, src, power, 1, 4) == BT_OK);
  CHECK(bt_set_microphones(ctx, sid, &mics[0][0], NM) == BT_OK);
  bt_trace_params p;
  bt_params_default(&p);
  p.max_order = 2;
  CHECK(bt_trace(ctx, sid, &p) == BT_OK);
  double level[NM][BT_MAX_BANDS], inten[NM][BT_MAX_BANDS];
  int32_t count[NM];
  bt_stats st;
  CHECK(bt_read_levels(ctx, sid, &level[0][0], &inten[0][0], count, &st) == BT_OK);
  CHECK(st.beams == 5120 && st.segments >= st.beams);
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < NM; m++) {
    double dx = (double)mics[m][0] - src[0], dy = (double)mics[m][1] - src[1];
    double dz = (double)mics[m][2] - src[2], dzi = (double)mics[m][2] + src[2];
    double d2 = dx * dx + dy * dy + dz * dz, di2 = dx * dx + dy * dy + dzi * dzi;
    CHECK(count[m] == 2);
    for (int b = 0; b < BT_MAX_BANDS; b++) {
      double expect = power[b] / (4.0 * pi * d2) + (double)refl[b] * power[b] / (4.0 * pi * di2);
      CHECK(fabs(inten[m][b] / expect - 1.0) < 1e-4);
      CHECK(fabs(level[m][b] - 10.0 * log10(expect / 1e-12)) < 1e-3);
    }
  }
  /* the same trace submitted asynchronously */
  CHECK(bt_submit(ctx, sid, &p) == BT_OK);
  CHECK(bt_wait(ctx, sid) == BT_OK);
  int32_t count2[NM];
  CHECK(bt_read_levels(ctx, sid, NULL, NULL, count2, NULL) == BT_OK);
  for (int m = 0; m < NM; m++) CHECK(count2[m] == count[m]);
  CHECK(bt_kernel_launches() > 0);
  CHECK(bt_unload_scene(ctx, sid) == BT_OK);
  CHECK(bt_destroy(ctx) == BT_OK);
}

int main(int argc, char **argv) {
  int expect_no_device = argc > 1 && strcmp(argv[1], "--no-device") == 0;
  int trace = argc > 1 && strcmp(argv[1], "--trace") == 0;
  /* layouts: every field of the parameters is 4 bytes wide, the stats are
   * 14 int64 counters then 3 doubles */
  CHECK(sizeof(bt_trace_params) == 4 * (1 + BT_MAX_BANDS + 1 + 1 + 2 + 1 + 1 + 1 + 1 + 1 + 1 + 3));
  CHECK(offsetof(bt_trace_params, air_atten_db_per_m) == 4);
  CHECK(offsetof(bt_trace_params, fault_test) == sizeof(bt_trace_params) - 4);
  CHECK(sizeof(bt_stats) == 8 * 17);
  CHECK(offsetof(bt_stats, trace_ms) == 8 * 14);

  bt_trace_params p;
  memset(&p, 0xff, sizeof(p));
  CHECK(bt_params_default(&p) == BT_OK);
  CHECK(p.max_order == 4 && p.tiles_x == 1 && p.tiles_y == 1 && p.precision == BT_PREC_MIXED);
  CHECK(p.t_eps_m == 1e-3f && p.watchdog_ms == 2000 && p.chunk_beams == 0 && p.queue_depth == 0);
  CHECK(p.leaf_size == 0 && p.beams_per_warp == 0 && p.fault_test == 0);
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
  if (trace) trace_ground_plane();
  if (failures == 0) printf("c_abi_check: ok\n");
  return failures == 0 ? 0 : 1;
}
