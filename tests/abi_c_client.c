/* A plain C99 client of include/rgs.h: it compiles with a C compiler (no C++ or CUDA
 * headers), links against librgs.so and exercises the entry points that need no device
 * (version, status strings, argument validation).  tests/test_abi.py builds and runs it. */
#include <stdio.h>
#include <string.h>

#include "rgs.h"

int main(void) {
    rgs_scene *scene = NULL;
    rgs_transport *transport = NULL;
    rgs_surfels surfels;
    rgs_transport_info info;
    int code;

    if (rgs_abi_version() != RGS_ABI_VERSION) return 1;
    for (code = RGS_OK; code <= RGS_ERR_STATE; ++code)
        if (!rgs_status_string((rgs_status)code) || !rgs_status_string((rgs_status)code)[0]) return 2;

    memset(&surfels, 0, sizeof surfels);
    surfels.n = 16;
    surfels.sh_degree = 2; /* every array left NULL */
    if (rgs_build_scene(&surfels, NULL, NULL, &scene) != RGS_ERR_ARG || scene != NULL) return 3;
    if (!strstr(rgs_last_error(), "NULL")) return 4;
    if (rgs_trace_transport(NULL, NULL, NULL, NULL, &transport) != RGS_ERR_ARG || transport != NULL) return 5;
    if (rgs_solve(NULL, NULL, 1, RGS_FP32, NULL, NULL, NULL) != RGS_ERR_ARG) return 6;
    if (rgs_adjoint(NULL, NULL, NULL, NULL, NULL, NULL) != RGS_ERR_ARG) return 7;
    if (rgs_transport_info_get(NULL, &info) != RGS_ERR_ARG) return 8;
    rgs_destroy_transport(NULL);
    rgs_destroy_scene(NULL);
    puts("rgs C client ok");
    return 0;
}
