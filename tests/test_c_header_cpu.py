"""include/shouji.h is a C header: a plain C11 program that includes it links
against libshouji.so and calls the entry points that need no GPU (size
helpers, status strings, argument checks)."""
import os
import shutil
import subprocess

import pytest

import paper_1809_07858_gb300 as sj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "shouji.h"

int main(void)
{
    if (shouji_packed_words(1, 100) != 100 * 64) return 1;
    if (shouji_nmask_words(1025, 100) != 2 * 100 * 32) return 2;
    if (strcmp(shouji_status_string(SHOUJI_EINVAL), shouji_status_string(SHOUJI_OK)) == 0) return 3;
    /* argument checks answer on the host, before any GPU work */
    if (shouji_filter(NULL, NULL, NULL, NULL, 100, 10, 5, NULL, NULL, NULL, NULL, NULL)
        != SHOUJI_EINVAL) return 4;
    if (shouji_magnet(NULL, NULL, NULL, NULL, 0, 10, 5, NULL, NULL, NULL, NULL, NULL)
        != SHOUJI_EINVAL) return 5;
    if (shouji_filter(NULL, NULL, NULL, NULL, 100, 0, 5, NULL, NULL, NULL, NULL, NULL)
        != SHOUJI_OK) return 6;
    if (shouji_compact_workspace_size(0) != 0) return 7;
    printf("ok %s\n", shouji_status_string(SHOUJI_ETIMEOUT));
    return 0;
}
"""


def test_header_compiles_as_c_and_links(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    lib_dir = os.path.dirname(sj.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", lib_dir, "-lshouji", "-Wl,-rpath," + lib_dir])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
