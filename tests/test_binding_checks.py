"""The Python binding rejects buffers whose size or dtype does not match what the
library will read or write, before any device call (CPU only: every case fails in
the argument checks, ahead of the device-pointer marshalling)."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ixp():
    import paper_2506_23058_gb300 as m
    m.load()
    return m


def test_partition_buffers(ixp):
    keys = torch.zeros(10, dtype=torch.int32)
    with pytest.raises(ValueError, match="payload"):
        ixp.partition(keys, ("lt", 0, 5), payload=torch.zeros(5, dtype=torch.float32))
    with pytest.raises(ValueError, match="out"):
        ixp.partition(keys, ("lt", 0, 5), out=torch.empty(9, dtype=torch.int32))
    with pytest.raises(ValueError, match="num_true"):
        ixp.partition(keys, ("lt", 0, 5), num_true=torch.empty(1, dtype=torch.int32))
    with pytest.raises(ValueError, match="flags"):
        ixp.partition(None, ("flags", 0, 0, torch.zeros(9, dtype=torch.uint8)), n=10)


def test_scatter_gather_buffers(ixp):
    idx = torch.zeros(8, dtype=torch.int64)
    with pytest.raises(ValueError, match="vals"):
        ixp.scatter(torch.zeros(4, 2), idx, torch.zeros(7, 2))
    with pytest.raises(ValueError, match="rows"):
        ixp.scatter(torch.zeros(4, 2, dtype=torch.float64), idx, torch.zeros(8, 2))
    with pytest.raises(ValueError, match="acc"):
        ixp.scatter_add_f64(torch.zeros(4, 2), idx, torch.zeros(8, 2))
    with pytest.raises(ValueError, match="out"):
        ixp.gather(torch.zeros(4, 2), idx, out=torch.zeros(8, 3))
    with pytest.raises(ValueError, match="out"):
        ixp.invert(idx, 10, out=torch.empty(9, dtype=torch.int64))


def test_check_buffers(ixp):
    z = torch.zeros(10, dtype=torch.int32)
    with pytest.raises(ValueError, match="keys"):
        ixp.check_filtpart(z, torch.zeros(9, dtype=torch.int32), part=("lt", 0, 1))
    with pytest.raises(ValueError, match="cls"):
        ixp.check_filtpart(z, cls=torch.zeros(10, dtype=torch.int32), v=3)
    with pytest.raises(ValueError, match="verdict"):
        ixp.check_range(z, out=torch.empty(5, dtype=torch.int64))


def test_scan_and_pairs_buffers(ixp):
    x = torch.zeros(10, dtype=torch.int32)
    with pytest.raises(ValueError, match="totals"):
        ixp.scan(x, out=torch.empty(10, dtype=torch.int64), totals=torch.empty(1, dtype=torch.int32))
    es = torch.zeros(10, dtype=torch.int64)
    with pytest.raises(ValueError, match="out_es"):
        ixp.smallest_pairs(es, es.clone(), 4, 10, out_es=torch.empty(9, dtype=torch.int64))
    with pytest.raises(ValueError, match="vals"):
        ixp.hist_min(torch.zeros(4, dtype=torch.int64), es, torch.zeros(9, dtype=torch.int64))


def test_sgm_scan_buffers(ixp):
    x = torch.zeros(10, dtype=torch.int32)
    with pytest.raises(ValueError, match="flags"):
        ixp.sgm_scan(torch.zeros(9, dtype=torch.uint8), x)
    with pytest.raises(ValueError, match="flags"):
        ixp.sgm_scan(torch.zeros(10, dtype=torch.int32), x)
    with pytest.raises(ValueError, match="out"):
        ixp.sgm_scan(torch.zeros(10, dtype=torch.uint8), x, out=torch.empty(9, dtype=torch.int64))
    with pytest.raises(ValueError, match="status"):
        ixp.sgm_scan(torch.zeros(10, dtype=torch.uint8), x, status=torch.zeros(1, dtype=torch.int64))


def test_scan_and_status_buffers(ixp):
    x = torch.zeros(10, dtype=torch.int32)
    with pytest.raises(ValueError, match="out"):
        ixp.scan(x, out=torch.empty(9, dtype=torch.int32))
    with pytest.raises(ValueError, match="status"):
        ixp.scan(x, status=torch.zeros(0, dtype=torch.int32))
    with pytest.raises(ValueError, match="status"):
        ixp.mkii(torch.zeros(2, dtype=torch.int64), 0, status=torch.zeros(1, dtype=torch.int64))
    with pytest.raises(ValueError, match="status"):
        ixp.gather(torch.zeros(4, 2), torch.zeros(3, dtype=torch.int64), status=torch.zeros(1, dtype=torch.uint8))


def test_filtpart_values_buffers(ixp):
    x = torch.zeros(10, 3, dtype=torch.int32)
    with pytest.raises(ValueError, match="type and shape"):
        ixp.check_filtpart_values(torch.zeros(10, 4, dtype=torch.int32), x)
    with pytest.raises(ValueError, match="type and shape"):
        ixp.check_filtpart_values(torch.zeros(10, 3, dtype=torch.float32), x)
    with pytest.raises(ValueError, match="multiple of 4"):
        ixp.check_filtpart_values(torch.zeros(10, 3, dtype=torch.uint8), torch.zeros(10, 3, dtype=torch.uint8))
    with pytest.raises(ValueError, match="keys"):
        ixp.check_filtpart_values(x, x, keys=torch.zeros(9, dtype=torch.int32))
    with pytest.raises(ValueError, match="cls"):
        ixp.check_filtpart_values(x, x, cls=torch.zeros(10, dtype=torch.int32), v=3)
