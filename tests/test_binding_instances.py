"""Argument marshalling of Scene.from_instances on the host (no GPU): the prototypes reach the C ABI
concatenated with vertex and triangle offsets that start at 0 and ascend, the instance maps as row-major
[n_inst][12] float32 rows, and the scene's sizes come back from st_scene_get_geometry.  A stand-in for the
library records what the binding passes."""
import ctypes as C

import numpy as np
import pytest


class _FakeLib:
    def __init__(self, nv, nt):
        self.seen = {}
        self.nv, self.nt = nv, nt

    @staticmethod
    def _arr(ptr, dtype, n):
        return np.ctypeslib.as_array(C.cast(ptr, C.POINTER(np.ctypeslib.as_ctypes_type(dtype))), shape=(n,)).copy()

    def st_scene_load_instances(self, h, n_proto, voff, pv, toff, pt, pm, n_inst, ip, xf, out):
        vo = self._arr(voff, np.int64, n_proto + 1)
        to = self._arr(toff, np.int64, n_proto + 1)
        self.seen.update(n_proto=n_proto, voff=vo, toff=to, pv=self._arr(pv, np.float32, 3 * vo[-1]),
                         pt=self._arr(pt, np.int32, 3 * to[-1]), pm=self._arr(pm, np.int32, to[-1]),
                         n_inst=n_inst, ip=self._arr(ip, np.int32, n_inst), xf=self._arr(xf, np.float32, 12 * n_inst))
        out._obj.value = 0x1000
        return 0

    def st_scene_get_geometry(self, h, nv, nt, *rest):
        nv._obj.value, nt._obj.value = self.nv, self.nt
        return 0


class _FakeCtx:
    h = None  # a closed context: the scene's destructor does nothing

    def __init__(self, L):
        self.L = L

    def _check(self, status):
        assert status == 0


def test_from_instances_marshalling():
    st = pytest.importorskip("paper_2602_19652_gb300")
    rng = np.random.default_rng(0)
    protos = []
    for nv, nt, mat in ((4, 2, 0), (6, 5, 3), (3, 1, 1)):
        protos.append((rng.normal(size=(nv, 3)), rng.integers(0, nv, (nt, 3)), np.full(nt, mat)))
    inst = np.array([2, 0, 1, 1], np.int32)
    X = rng.normal(size=(4, 3, 4))
    nv = sum(len(protos[q][0]) for q in inst)
    nt = sum(len(protos[q][1]) for q in inst)
    L = _FakeLib(nv, nt)
    sc = st.Scene.from_instances(_FakeCtx(L), protos, inst, X)
    s = L.seen
    assert s["n_proto"] == 3 and s["n_inst"] == 4
    assert list(s["voff"]) == [0, 4, 10, 13] and list(s["toff"]) == [0, 2, 7, 8]
    assert np.array_equal(s["pv"].reshape(-1, 3), np.concatenate([p[0] for p in protos]).astype(np.float32))
    assert np.array_equal(s["pt"].reshape(-1, 3), np.concatenate([p[1] for p in protos]).astype(np.int32))
    assert np.array_equal(s["pm"], np.concatenate([p[2] for p in protos]).astype(np.int32))
    assert np.array_equal(s["ip"], inst)
    assert np.array_equal(s["xf"].reshape(4, 3, 4), X.astype(np.float32))  # [A | b] rows, row-major
    assert (sc.n_verts, sc.n_tris, sc.n_inst, sc.n_obj) == (nv, nt, 4, 4)
