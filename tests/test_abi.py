"""The C-ABI library builds, loads without a GPU and exports every entry point of include/fhr.h."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fhr.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fhr_[a-z_0-9]+)\s*\(", src)))


def test_header_names_match_binding():
    from paper_2410_22500_gb300 import fhr

    assert sorted(fhr.ENTRY_POINTS) == _declared()


def test_library_exports_every_entry_point(lib_path):
    L = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(fhr_[a-z_0-9]+)", out))
    assert set(_declared()) <= exported


def test_version_and_no_device_error(lib_path):
    import torch
    from paper_2410_22500_gb300 import fhr

    L = fhr.load()
    assert L.fhr_version().startswith(b"libfhr")
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert L.fhr_create(ctypes.byref(h), 0, None) == fhr.ERR_ARG
        assert not h.value


def test_struct_layout_matches_c(tmp_path):
    # compile a probe with the system C compiler against the header and compare
    # sizes / offsets with the ctypes mirrors
    from paper_2410_22500_gb300 import fhr

    src = tmp_path / "probe.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "fhr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(fhr_norm_params), sizeof(fhr_nmf_params), sizeof(fhr_geom),
         sizeof(fhr_mbir_params), sizeof(fhr_pipeline_params));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", offsetof(fhr_nmf_params, seed), offsetof(fhr_mbir_params, sigma_v),
         offsetof(fhr_pipeline_params, geom), offsetof(fhr_pipeline_params, mbir),
         offsetof(fhr_pipeline_params, host_io), offsetof(fhr_nmf_params, mlp_params), sizeof(fhr_mlp_dims));
  printf("%zu %zu %zu\n", offsetof(fhr_nmf_params, kmeans_samples), offsetof(fhr_nmf_params, kmeans_iters),
         offsetof(fhr_pipeline_params, recon));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(fhr_problem), offsetof(fhr_problem, sino), offsetof(fhr_problem, sigma_x),
         sizeof(fhr_batch_params), offsetof(fhr_batch_params, tile), offsetof(fhr_batch_params, vw));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes, offs, km, batch = [list(map(int, l.split()))
                          for l in subprocess.check_output([str(exe)], text=True).splitlines()]
    assert sizes == [ctypes.sizeof(t) for t in (fhr.NormParams, fhr.NmfParams, fhr.Geom, fhr.MbirParams,
                                                 fhr.PipelineParams)]
    assert offs == [fhr.NmfParams.seed.offset, fhr.MbirParams.sigma_v.offset, fhr.PipelineParams.geom.offset,
                    fhr.PipelineParams.mbir.offset, fhr.PipelineParams.host_io.offset, fhr.NmfParams.mlp_params.offset,
                    ctypes.sizeof(fhr.MlpDims)]
    assert km == [fhr.NmfParams.kmeans_samples.offset, fhr.NmfParams.kmeans_iters.offset,
                  fhr.PipelineParams.recon.offset]
    assert batch == [ctypes.sizeof(fhr.Problem), fhr.Problem.sino.offset, fhr.Problem.sigma_x.offset,
                     ctypes.sizeof(fhr.BatchParams), fhr.BatchParams.tile.offset, fhr.BatchParams.vw.offset]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2410_22500_gb300 import fhr

    monkeypatch.setattr(fhr, "_lib", None)
    monkeypatch.setattr(fhr, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        fhr.load()
