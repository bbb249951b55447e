"""Seeded inputs of the controller network (weights and feature batches) and
the BF16 storage format (round-to-nearest-even of FP32, as 16-bit patterns).
No arithmetic of the network itself lives here."""
import numpy as np

N_IN, N_HID, N_OUT = 16, 64, 2
N_PARAMS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_OUT * N_HID + N_OUT


def init_weights(seed: int) -> np.ndarray:
    """Scaled-normal initial weights (1/sqrt(fan-in)), zero biases, flat FP32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4D4C50]))
    parts = [rng.normal(0.0, 1.0 / np.sqrt(N_IN), N_HID * N_IN), np.zeros(N_HID),
             rng.normal(0.0, 1.0 / np.sqrt(N_HID), N_HID * N_HID), np.zeros(N_HID),
             rng.normal(0.0, 1.0 / np.sqrt(N_HID), N_OUT * N_HID), np.zeros(N_OUT)]
    return np.concatenate(parts).astype(np.float32)


def features(seed: int, batch: int) -> np.ndarray:
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x464541]))
    return rng.normal(0.0, 1.0, (batch, N_IN)).astype(np.float32)


def bf16_bits(w) -> np.ndarray:
    """Round FP32 values to BF16 (nearest, ties to even) and return the bit patterns."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    return r.astype(np.uint16)


def bf16_values(bits) -> np.ndarray:
    """FP32 values of BF16 bit patterns."""
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)
