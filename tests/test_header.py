"""The public header compiles as C and as C++ with the host compilers (no
CUDA headers needed by a consumer of the C ABI)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("cc,lang", [("gcc", "c"), ("g++", "c++")])
def test_header_compiles(tmp_path, cc, lang):
    exe = shutil.which(cc)
    if exe is None:
        pytest.skip(f"no {cc}")
    src = tmp_path / ("t.c" if lang == "c" else "t.cpp")
    src.write_text('#include "mqo.h"\nint main(void) { mqo_params p; (void)p; return (int)MQO_OK; }\n')
    subprocess.run([exe, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-fsyntax-only", str(src)],
                   check=True)
