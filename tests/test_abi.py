"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/lic.h declares, and its host-built entropy tables equal the
oracle's bit for bit (two independent FP64 implementations of the same
definitions: the factorized bottleneck of Ballé 2018 app. 6.1 and the
Gaussian conditional with 64 scales)."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lic_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_function():
    path = lic.LIB_PATH
    assert os.path.exists(path), "liblic.so must be built"
    out = subprocess.check_output(["nm", "-D", "--defined-only", path], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    decl = declared_functions()
    assert decl, "no declarations parsed"
    missing = decl - exported
    assert not missing, missing
    L = lic.lib()
    for name in decl:
        assert hasattr(L, name)
    assert set(lic.EXPORTED) <= decl


def test_strerror():
    L = lic.lib()
    assert L.lic_strerror(0) == b"ok"
    assert b"corrupt" in L.lic_strerror(-4)


@pytest.mark.parametrize("kind,N,M", [(0, 32, 64), (1, 64, 96)])
def test_host_tables_match_oracle_bit_exactly(kind, N, M):
    W = synth.make_weights(kind, N, M)
    med, lo, hi, start, cdf = lic.build_tables(W, gauss=(kind == 1))
    omed, otabs = O.eb_tables(W)
    assert np.array_equal(med.view(np.uint32), omed.view(np.uint32))
    tabs = list(otabs)
    if kind == 1:
        tabs += O.gauss_tables()
    assert len(lo) == len(tabs)
    for t, ot in enumerate(tabs):
        assert (lo[t], hi[t]) == (ot.lo, ot.hi)
        n = ot.n
        assert np.array_equal(cdf[start[t]:start[t] + n + 1], ot.cdf), t


def test_scale_table_matches_oracle():
    assert np.array_equal(lic.scale_table().view(np.uint32), O.scale_table().view(np.uint32))


def test_decoded_shape_reads_oracle_container():
    buf = O.pack_frame(1, 128, 192, 721, 1279, 768, 1280, 16, [np.zeros(64, np.uint16)])
    assert lic.decoded_shape(buf) == (1, 721, 1279)
    with pytest.raises(lic.LicError):
        lic.decoded_shape(b"XXXX" + buf[4:])


def test_student_create_validates_arguments_before_device_work():
    """lic_student_create refuses bad options and missing or mis-sized
    parameters with LIC_E_INVALID_ARG (no device needed to reach the check)."""
    W = synth.make_student_weights()
    bad_opts = (dict(max_batch=0), dict(max_batch=lic.STUDENT_MAX_BATCH + 1), dict(crop=40), dict(crop=16),
                dict(lr=0.0), dict(beta1=1.0), dict(eps=0.0), dict(precision=lic.FP8), dict(halo=-1),
                dict(halo=9))
    for kw in bad_opts:
        with pytest.raises(lic.LicError) as e:
            lic.Student(W, **kw)
        assert e.value.code == lic.E_INVALID_ARG, kw
    missing = {k: v for k, v in W.items() if k != "student.deconv2.bias"}
    wrong = dict(W)
    wrong["student.deconv1.weight"] = W["student.deconv1.weight"][:32]
    for w in (missing, wrong):
        with pytest.raises(lic.LicError) as e:
            lic.Student(w)
        assert e.value.code == lic.E_INVALID_ARG
    with pytest.raises(lic.LicError):
        lic.Student(W, M=100)
