/* A plain C program against the C ABI in qld.h: it must compile as C99 and
 * link to libqld.so. It calls only the entry points that answer before
 * touching a device (argument checks, sizes, status strings), so it runs on
 * a machine without a GPU, and prints "ok" when every answer is right. */
#include <stdio.h>
#include <string.h>

#include "qld.h"

static int fails = 0;

static void check(int cond, const char* what) {
    if (!cond) {
        printf("failed: %s\n", what);
        ++fails;
    }
}

int main(void) {
    check(qld_create(0, 16, 8, QLD_U16) == NULL && qld_last_error() == QLD_E_INVAL, "create rejects H = 0");
    check(qld_create(16, 16, 6, QLD_U16) == NULL && qld_last_error() == QLD_E_INVAL, "create rejects N mod 4 != 0");
    check(qld_create_band(16, 16, 8, QLD_U16, 12, 8) == NULL && qld_last_error() == QLD_E_INVAL,
          "band must lie inside the frame");
    check(qld_create_band(16, 15, 8, QLD_P12, 1, 2) == NULL && qld_last_error() == QLD_E_INVAL,
          "packed band must start on a pixel pair");
    /* ring of 64 16-KiB slots, two int32 sum planes, 64 float2 twiddles in 512 bytes */
    check(qld_footprint_bytes(128, 128, 64, QLD_U8) == 64LL * 16384 + 2LL * 4 * 16384 + 512, "footprint");
    check(qld_push_frames(NULL, NULL, 0, NULL) == QLD_E_INVAL, "push to no context");
    check(qld_fft_bin(NULL, 0, NULL) == QLD_E_INVAL, "DFT bin of no context");
    check(qld_frames_pushed(NULL) == -1, "frames pushed of no context");
    check(strncmp(qld_strerror(QLD_E_NOT_READY), "window not full", 15) == 0, "status string");
    check(qld_server_create(0, 1) == NULL && qld_last_error() == QLD_E_INVAL, "server rejects a zero budget");
    check(qld_server_num_shapes() >= 1, "server launch shapes");
    check(qld_server_set_shape(NULL, 0) == QLD_E_INVAL, "shape of no server");
    puts(fails ? "FAIL" : "ok");
    return fails;
}
