"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every entry point that include/dsps.h declares;
the oracle and the CUDA path share no code."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dsps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsps_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dsps_create", "dsps_destroy", "dsps_filters_add", "dsps_weights", "dsps_photometry",
              "dsps_photometry_vjp", "dsps_submit", "dsps_poll", "dsps_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2112_06830_gb300 import dsps
    lib = dsps.load()
    assert os.path.exists(dsps.library_path())
    raw = ctypes.CDLL(dsps.library_path())
    for n in _declared():
        assert hasattr(raw, n), n
    assert lib.dsps_strerror(0) == b"ok"
    assert b"budget" in lib.dsps_strerror(-2)


def test_default_opts():
    from paper_2112_06830_gb300 import dsps
    o = dsps.dsps_default_opts()
    assert (o.om0, o.w0, o.h) == (0.3, -1.0, 0.7)
    assert o.max_chunk == 262144 and o.z_max == 10.0 and o.n_streams == 4
    assert (o.dust_bump, o.dust_law, o.dust_agedep) == (0, dsps.DSPS_DUST_POWERLAW, 0)
    assert (o.dust_agedep_x0, o.dust_agedep_h) == (7.0, 0.1)
    assert (o.mdf_mean, o.mdf_terf_x0, o.mdf_terf_h) == (dsps.DSPS_MDF_MEAN_LINEAR, 9.0, 0.5)
    assert o.agedep_fused == 1


def test_struct_layouts_match_the_header():
    """The ctypes mirrors of dsps_grid / dsps_opts end with the fields the
    header declares last (a mismatch would shift every later field)."""
    import re
    from paper_2112_06830_gb300 import dsps
    hdr = open(os.path.join(ROOT, "include", "dsps.h")).read()
    for cname, pyc in (("dsps_grid", dsps.dsps_grid), ("dsps_opts", dsps.dsps_opts),
                       ("dsps_line_spec", dsps.dsps_line_spec), ("dsps_hist_spec", dsps.dsps_hist_spec)):
        body = re.search(r"typedef struct \{([^{}]*)\} " + cname + ";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            decl = re.sub(r"\bconst\b|\*", " ", decl)
            parts = decl.split()
            names += [n.strip() for n in " ".join(parts[1:]).split(",")]
        assert [f[0] for f in pyc._fields_] == names, cname


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    from paper_2112_06830_gb300 import dsps, synth
    g = synth.make_ssp(synth.GridSpec(4, 2, 16, 1e3, 1e4), 0)
    with pytest.raises(dsps.DSPSError) as ei:
        dsps.Context(g)
    assert ei.value.code in (dsps.DSPS_ERR_CUDA, dsps.DSPS_ERR_UNSUPPORTED)


def test_oracle_and_cuda_path_share_no_code():
    csrc = os.path.join(ROOT, "paper_2112_06830_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    orc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "#include \"" not in orc
    for f in ("dsps.py", "build.py", "synth.py", "autograd.py", "serve.py"):
        p = os.path.join(ROOT, "paper_2112_06830_gb300", f)
        if os.path.exists(p):
            assert "import oracle" not in open(p).read() and "from oracle" not in open(p).read(), f
