"""Host side of the autotuner (no device work): the table that later plans
consult, read from the TFFT_TUNE_CACHE file, matched on (n, dtype, checksum
mode, precision) with the nearest batch in log2, and the options the tuner
refuses.  The timing itself runs on the GPU (test_gpu_tune.py)."""
import pytest

import paper_2405_02520_gb300 as t

C64, C128, ON, OFF = t.TFFT_C64, t.TFFT_C128, t.TFFT_ABFT_TWO_SIDED, t.TFFT_ABFT_OFF


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("TFFT_TUNE_CACHE", str(path))
    t.tfft_tune_clear()
    yield path
    monkeypatch.delenv("TFFT_TUNE_CACHE")
    t.tfft_tune_clear()


def test_no_entry_no_configuration(cache):
    assert t.tfft_tune_lookup(1 << 16, 64, C64, ON) is None


def test_entries_matched_on_transform_and_nearest_batch(cache):
    cache.write_text("tfft-tune-1 65536 64 0 2 0 2 9 512 1.5\n"
                     "tfft-tune-1 65536 4096 0 2 0 2 10 256 1.2\n"
                     "tfft-tune-1 65536 64 0 0 0 2 8 256 1.0\n"
                     "tfft-tune-1 1048576 1 1 2 0 3 0 256 9.0\n")
    t.tfft_tune_clear()
    assert t.tfft_tune_lookup(1 << 16, 64, C64, ON) == (2, 9, 512)
    assert t.tfft_tune_lookup(1 << 16, 128, C64, ON) == (2, 9, 512)        # log2 distance 1 against 5
    assert t.tfft_tune_lookup(1 << 16, 2048, C64, ON) == (2, 10, 256)
    assert t.tfft_tune_lookup(1 << 16, 64, C64, OFF) == (2, 8, 256)         # the checksum mode is part of the key
    assert t.tfft_tune_lookup(1 << 16, 64, C128, ON) is None                # and the dtype
    assert t.tfft_tune_lookup(1 << 16, 64, C64, ON, precision=t.TFFT_PREC_BF16X3) is None
    assert t.tfft_tune_lookup(1 << 20, 7, C128, ON) == (3, 0, 256)          # three passes: no first factor
    assert t.tfft_tune_lookup(1 << 15, 64, C64, ON) is None


def test_equal_distance_takes_the_later_entry(cache):
    cache.write_text("tfft-tune-1 4096 16 0 2 0 1 0 256 0.5\n"
                     "tfft-tune-1 4096 64 0 2 0 2 6 256 0.4\n")
    t.tfft_tune_clear()
    assert t.tfft_tune_lookup(4096, 32, C64, ON) == (2, 6, 256)


def test_malformed_and_out_of_range_lines_are_skipped(cache):
    cache.write_text("not a tuning line\n"
                     "tfft-tune-2 65536 64 0 2 0 2 9 512 1.5\n"      # another format version
                     "tfft-tune-1 65536 64 0 2 0 4 9 512 1.5\n"      # four passes
                     "tfft-tune-1 65536 64 0 2 0 2 9 384 1.5\n"      # 384 threads
                     "tfft-tune-1 65535 64 0 2 0 2 9 512 1.5\n"      # n not a power of two
                     "tfft-tune-1 65536 64 0 2\n"                    # short
                     "tfft-tune-1 65536 64 0 2 0 1 0 256 2.0\n")
    t.tfft_tune_clear()
    assert t.tfft_tune_lookup(1 << 16, 64, C64, ON) == (1, 0, 256)


def test_clear_rereads_the_file(cache):
    cache.write_text("tfft-tune-1 256 8 0 2 0 1 0 256 0.1\n")
    t.tfft_tune_clear()
    assert t.tfft_tune_lookup(256, 8, C64, ON) == (1, 0, 256)
    cache.write_text("")
    assert t.tfft_tune_lookup(256, 8, C64, ON) == (1, 0, 256)               # the table is kept in memory
    t.tfft_tune_clear()
    assert t.tfft_tune_lookup(256, 8, C64, ON) is None


def test_no_cache_file_no_entries(monkeypatch):
    monkeypatch.delenv("TFFT_TUNE_CACHE", raising=False)
    t.tfft_tune_clear()
    assert t.tfft_tune_lookup(1 << 16, 64, C64, ON) is None


@pytest.mark.parametrize("forced", [{"force_passes": 2}, {"first_pass_log2": 8}, {"tile_threads": 256}])
def test_autotune_refuses_options_that_fix_the_configuration(forced):
    with pytest.raises(t.TfftError) as e:
        t.tfft_autotune(1 << 16, 64, C64, ON, 16, 32, reps=1, **forced)
    assert e.value.code == -1


@pytest.mark.parametrize("reps", [0, 1001])
def test_autotune_refuses_repetition_counts_out_of_range(reps):
    with pytest.raises(t.TfftError) as e:
        t.tfft_autotune(1 << 16, 64, C64, ON, 16, 32, reps=reps)
    assert e.value.code == -1


@pytest.mark.parametrize("threads", [128, 384, 1024, -256])
def test_tile_threads_other_than_256_or_512_rejected_before_device_work(threads):
    with pytest.raises(t.TfftError) as e:
        t.tfft_plan_ex(1 << 16, 64, C64, ON, tile_threads=threads)
    assert e.value.code == -1
