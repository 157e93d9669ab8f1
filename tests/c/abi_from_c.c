/* A plain C program against include/mms.h and libmms.so: the boundary needs
 * no C++, CUDA or Python types.  Only host-side calls (version, variant
 * counts, argument refusals), so it runs without a GPU.  With the arguments
 * "gpu PATH VARIANT" (on a GPU) it also checks that AUTO and the default
 * variant of the box of radius 2 are those of the library's built-in tuned
 * table for the device, with nothing registered by the caller. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mms.h"

static int fails = 0;

static void expect(int cond, const char *what)
{
    if (!cond) {
        fprintf(stderr, "FAIL: %s (last error: %s)\n", what, mms_last_error());
        ++fails;
    }
}

int main(int argc, char **argv)
{
    float c[27] = {0};
    float buf[64] = {0};
    mms_stencil_desc d;
    mms_wave_desc w;

    expect(strstr(mms_version(), "sm_103a") != NULL, "version names the target");
    expect(mms_num_variants(MMS_STAR, 4, MMS_PATH_CUDA_CORE) > 0, "star r=4 has CUDA-core variants");
    expect(mms_num_variants(MMS_BOX, 9, MMS_PATH_CUDA_CORE) == 0, "no variants for radius 9");
    expect(mms_auto_path(MMS_STAR, 4, 0) == MMS_PATH_NAIVE, "unaligned input takes the naive path");
    expect(mms_stencil_apply(MMS_STAR, 5, c, buf, buf + 32, 8, 8, 8, NULL) == MMS_E_ARG, "radius 5 refused");
    expect(mms_stencil_apply(MMS_STAR, 4, c, buf, buf, 0, 8, 8, NULL) == MMS_OK, "empty interior is a no-op");

    memset(&d, 0, sizeof d);
    d.shape = MMS_BOX;
    d.radius = 1;
    d.coeffs = c;
    d.nx = d.ny = d.nz = 8;
    d.in_pitch_y = -4;
    expect(mms_stencil_apply_ex(&d, buf, buf + 32, NULL) == MMS_E_ARG, "negative pitch refused");

    memset(&w, 0, sizeof w);
    w.nx = w.ny = w.nz = 8;
    w.radius = 4;
    w.nshots = 65;
    w.rec_z = -1;
    expect(mms_wave_step(&w, c, buf, buf, buf + 32, buf, NULL, NULL) == MMS_E_ARG, "65 shots refused");
    expect(strlen(mms_last_error()) > 0, "refusals leave a message");

    if (argc > 3 && strcmp(argv[1], "gpu") == 0) {
        const int want_path = atoi(argv[2]), want_variant = atoi(argv[3]);
        expect(mms_auto_path(MMS_BOX, 2, 1) == want_path, "AUTO of the box r=2 follows the built-in table");
        expect(mms_default_variant(MMS_BOX, 2, want_path, 512, 512, 512) == want_variant,
               "default variant of the box r=2 follows the built-in table");
    }

    if (fails == 0) printf("ok\n");
    return fails;
}
