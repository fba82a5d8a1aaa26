"""Host logic of the engine that needs no GPU: which sorted-pair struct a
reverse pass receives.  The library's compute calls are replaced by no-ops;
only the buffers (on the CPU) and the structs are real."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def engine(monkeypatch):
    from paper_2602_00395_gb300 import engine as E
    from paper_2602_00395_gb300 import gs3dtr as G
    G.load()
    for name in ("gs_bin_sort", "gs_raster_fwd"):
        monkeypatch.setattr(G, name, lambda *a, **k: None)
    return E.TRStep(64, 0, 1, 32, 32, nu=0, device="cpu", capacity=1024)


def test_reverse_passes_get_the_block_masks_only_after_a_forward_pass(engine):
    """The forward pass writes the block masks of the current sort; a reverse
    pass gets them only between that forward pass and the next bin-sort (else
    NULL, and it tests the footprints itself)."""
    e = engine
    assert e.sorted().masks == e.masks.data_ptr()  # the forward pass always gets the buffer
    assert e.sorted_rev().masks is None  # nothing written yet
    e.bin_sort()
    assert e.sorted_rev().masks is None
    e.raster_fwd()
    assert e.sorted_rev().masks == e.masks.data_ptr()
    e.bin_sort()  # new pairs: the masks no longer describe them
    assert e.sorted_rev().masks is None
    e.raster_fwd()
    e._alloc_pairs(2048)  # a larger pair buffer: a new, unwritten mask buffer
    assert e.sorted_rev().masks is None and e.masks.numel() == 2048
