"""The C ABI used from C: include/npcf.h compiles as C99, and a C program linked against
libnpcf.so gets the documented defaults and the documented host-side argument errors
(no GPU needed: these calls return before any device work)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "npcf.h"

static int fails = 0;
#define EXPECT(c) do { if (!(c)) { printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); ++fails; } } while (0)

int main(void)
{
    npcf_opts o;
    memset(&o, 0x7f, sizeof o);
    npcf_default_opts(&o);
    EXPECT(o.precision == NPCF_FP32 && o.periodic == 1 && o.bin_order == NPCF_BINS_LE);
    EXPECT(o.sync_check == 1 && o.timing == 0);
    EXPECT(o.remove_self == 0 && o.parity == NPCF_PARITY_ALL);

    EXPECT(npcf_compute(NULL, NULL, NULL, 0, NULL, 0, 0, NULL) == NPCF_ERR_ARG);
    EXPECT(strstr(npcf_last_error(), "NULL") != NULL);

    npcf_plan_t plan = NULL;
    const double edges[3] = {0.1, 0.2, 0.3};
    const double edges5[6] = {0.05, 0.1, 0.15, 0.2, 0.25, 0.3};
    const double box[5] = {1.0, 1.0, 1.0, 1.0, 1.0};
    EXPECT(npcf_plan_create(&plan, 5, 3, 2, edges, 2, box, &o) == NPCF_ERR_UNSUPPORTED);
    EXPECT(plan == NULL);
    EXPECT(npcf_plan_create(&plan, 3, 6, 2, edges, 2, box, NULL) == NPCF_ERR_UNSUPPORTED);
    const double bad_edges[3] = {0.2, 0.1, 0.3};
    EXPECT(npcf_plan_create(&plan, 3, 3, 2, bad_edges, 2, box, NULL) == NPCF_ERR_ARG);
    EXPECT(strlen(npcf_last_error()) > 0);
    /* the options are validated on the host, before any device work */
    o.remove_self = 2;
    EXPECT(npcf_plan_create(&plan, 3, 3, 2, edges, 2, box, &o) == NPCF_ERR_ARG);
    npcf_default_opts(&o);
    o.parity = 5;
    EXPECT(npcf_plan_create(&plan, 3, 3, 2, edges, 2, box, &o) == NPCF_ERR_ARG);
    o.parity = NPCF_PARITY_ODD; /* N=3 has no odd-parity components */
    EXPECT(npcf_plan_create(&plan, 3, 3, 2, edges, 2, box, &o) == NPCF_ERR_UNSUPPORTED);
    npcf_default_opts(&o);
    o.precision = NPCF_MIXED_TF32X3; /* split precision: the D=2 4PCF (both) and the D=3 5PCF (BF16x3) */
    EXPECT(npcf_plan_create(&plan, 3, 3, 2, edges, 2, box, &o) == NPCF_ERR_UNSUPPORTED);
    EXPECT(npcf_plan_create(&plan, 3, 5, 2, edges5, 5, box, &o) == NPCF_ERR_UNSUPPORTED);
    o.precision = NPCF_MIXED_BF16X3;
    EXPECT(npcf_plan_create(&plan, 3, 4, 2, edges5, 5, box, &o) == NPCF_ERR_UNSUPPORTED);
    EXPECT(plan == NULL);
    npcf_plan_destroy(NULL);
    printf("%d failures\n", fails);
    return fails != 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_2106_10278_gb300 import build

    return os.path.dirname(build.build())


def test_header_is_c99():
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c",
                    os.path.join(ROOT, "include", "npcf.h")], check=True)


def test_c_program_links_and_gets_documented_errors(libdir, tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lnpcf", f"-Wl,-rpath,{libdir}"], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "0 failures" in res.stdout
